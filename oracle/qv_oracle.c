/*
 * qv_oracle.c -- plain, slow FP64 CPU reference for QV-Tree Search.
 *
 * Test infrastructure: only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg use this file.  Every function follows one
 * passage of the paper (cited beside it) without blocking, fusion or
 * reordering beyond what that passage states.  Where the paper is silent the
 * reading taken is stated in the comment.
 */
#include "qv_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const int DR[4] = {-1, 0, 1, 0};  /* N E S W: row step */
static const int DC[4] = {0, 1, 0, -1};  /*          col step */

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (timing single- and
 * multi-threaded runs of the same process). */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static int is_free(const or_problem *p, int r, int c) {
    if (r < 0 || r >= p->H || c < 0 || c >= p->W) return 0;  /* outside = occupied */
    return p->occ[r * p->W + c] == 0;
}

/* Stage reward r(y) of arriving in y.  Reading of the paper's r(x) (Sec. V)
 * with this workload's values: +100 at the goal, -1 - c(y) elsewhere.      */
static double stage_reward(const or_problem *p, int y) {
    if (y == p->goal) return 100.0;
    return -1.0 - (p->cost ? p->cost[y] : 0.0);
}

/* Observation label: nearest beacon by Manhattan distance within range,
 * ties to the lower id; none in range -> the null observation B.          */
void or_labels(const or_problem *p, int *label) {
    for (int r = 0; r < p->H; ++r)
        for (int c = 0; c < p->W; ++c) {
            int best = p->B, bestd = 1 << 30;
            for (int k = 0; k < p->B; ++k) {
                int br = p->beacon[k] / p->W, bc = p->beacon[k] % p->W;
                int d = abs(br - r) + abs(bc - c);
                if (d <= p->range && d < bestd) { best = k; bestd = d; }
            }
            label[r * p->W + c] = best;
        }
}

/* T(x, a, .) -- Sec. II dynamics with Eq. 10: the mass aimed at an occupied
 * (or outside) cell y is added to T(x, a, x).  Free-space kernel T': the
 * intended move w.p. 1 - 2 eps, each perpendicular move w.p. eps; stay is
 * deterministic.  Occupied cells and the goal are absorbing.              */
int or_transition_row(const or_problem *p, int x, int a, int *y, double *pr) {
    int n = 0;
    if (p->occ[x] || x == p->goal || a == 4) {
        y[0] = x; pr[0] = 1.0;
        return 1;
    }
    int r = x / p->W, c = x % p->W;
    int dirs[3] = {a, (a + 1) % 4, (a + 3) % 4};
    double w[3] = {1.0 - 2.0 * p->slip, p->slip, p->slip};
    for (int i = 0; i < 3; ++i) {
        int rr = r + DR[dirs[i]], cc = c + DC[dirs[i]];
        int t = is_free(p, rr, cc) ? rr * p->W + cc : x;   /* Eq. 10 */
        int j;
        for (j = 0; j < n; ++j)
            if (y[j] == t) { pr[j] += w[i]; break; }
        if (j == n) { y[n] = t; pr[n] = w[i]; ++n; }
    }
    return n;
}

/* R(x, a) = sum_y T(x, a, y) r(y) (Sec. V, the reward through the transition
 * model); the goal and occupied cells earn nothing.                       */
void or_reward_table(const or_problem *p, double *R) {
    int n = p->H * p->W;
    for (int a = 0; a < OR_NUM_ACTIONS; ++a)
        for (int x = 0; x < n; ++x) {
            double s = 0.0;
            if (!p->occ[x] && x != p->goal) {
                int y[3]; double pr[3];
                int m = or_transition_row(p, x, a, y, pr);
                for (int j = 0; j < m; ++j) s += pr[j] * stage_reward(p, y[j]);
            }
            R[a * n + x] = s;
        }
}

/* O(x', z): alpha for the cell's own label, eta = (1 - alpha)/B otherwise. */
double or_obs_lik(const or_problem *p, const int *label, int x, int z) {
    double eta = (1.0 - p->acc) / (double)p->B;
    return label[x] == z ? p->acc : eta;
}

/* MDP value iteration (Sec. V-B baseline; Bellman operator of Eq. 2 with a
 * known state): V_{k+1}(x) = max_a [R(x,a) + gamma sum_y T(x,a,y) V_k(y)],
 * Jacobi sweeps from V_0 = 0, V(goal) = 0, occupied cells 0.  The result Q is
 * R + gamma T V_final, the QMDP alpha-vectors used at the leaves (Eq. 4). */
int or_value_iteration(const or_problem *p, double tol, int max_sweeps, int truncated,
                       double *V, double *Q, int *sweeps, double *residual,
                       double *residual_hist) {
    int n = p->H * p->W;
    double *R = (double *)malloc(sizeof(double) * 5 * n);
    double *Vn = (double *)malloc(sizeof(double) * n);
    or_reward_table(p, R);
    for (int x = 0; x < n; ++x) V[x] = 0.0;
    int k = 0, status = 1;
    double res = 0.0;
    int limit = truncated > 0 ? truncated : max_sweeps;
    while (k < limit) {
        res = 0.0;
        for (int x = 0; x < n; ++x) {
            if (p->occ[x] || x == p->goal) { Vn[x] = 0.0; continue; }
            double best = -HUGE_VAL;
            for (int a = 0; a < OR_NUM_ACTIONS; ++a) {
                int y[3]; double pr[3];
                int m = or_transition_row(p, x, a, y, pr);
                double s = 0.0;
                for (int j = 0; j < m; ++j) s += pr[j] * V[y[j]];
                double q = R[a * n + x] + p->gamma * s;
                if (q > best) best = q;
            }
            Vn[x] = best;
            double d = fabs(best - V[x]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * n);
        if (residual_hist) residual_hist[k] = res;
        ++k;
        if (truncated <= 0 && res < tol) { status = 0; break; }
    }
    if (truncated > 0) status = 0;
    for (int a = 0; a < OR_NUM_ACTIONS; ++a)
        for (int x = 0; x < n; ++x) {
            if (p->occ[x] || x == p->goal) { Q[a * n + x] = 0.0; continue; }
            int y[3]; double pr[3];
            int m = or_transition_row(p, x, a, y, pr);
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += pr[j] * V[y[j]];
            Q[a * n + x] = R[a * n + x] + p->gamma * s;
        }
    *sweeps = k;
    *residual = res;
    free(R); free(Vn);
    return status;
}

/* Numerator of Eq. 3: bbar(x') = sum_x T(x, a, x') b(x).  A belief carries
 * no mass on occupied cells (Sec. II); values stored there are read as 0. */
void or_predict(const or_problem *p, const double *b, int a, double *bbar) {
    int n = p->H * p->W;
    for (int x = 0; x < n; ++x) bbar[x] = 0.0;
    for (int x = 0; x < n; ++x) {
        if (p->occ[x]) continue;
        int y[3]; double pr[3];
        int m = or_transition_row(p, x, a, y, pr);
        for (int j = 0; j < m; ++j) bbar[y[j]] += pr[j] * b[x];
    }
}

/* Denominator of Eq. 3: P(z | b, a) = sum_x' O(x', z) bbar(x'), z = 0..B. */
void or_obs_marginal(const or_problem *p, const int *label, const double *bbar, double *P) {
    int n = p->H * p->W;
    for (int z = 0; z <= p->B; ++z) {
        double s = 0.0;
        for (int x = 0; x < n; ++x) s += or_obs_lik(p, label, x, z) * bbar[x];
        P[z] = s;
    }
}

/* Eq. 3: Phi(b, a, z)(x') = O(x', z) bbar(x') / P(z | b, a).              */
double or_correct(const or_problem *p, const int *label, const double *bbar, int z, double *bout) {
    int n = p->H * p->W;
    double pz = 0.0;
    for (int x = 0; x < n; ++x) pz += or_obs_lik(p, label, x, z) * bbar[x];
    for (int x = 0; x < n; ++x) bout[x] = or_obs_lik(p, label, x, z) * bbar[x] / pz;
    return pz;
}

/* R(b, a) = sum_x R(x, a) b(x)  (Sec. III, after Eq. 2).                   */
double or_belief_reward(const or_problem *p, const double *R, const double *b, int a) {
    int n = p->H * p->W;
    double s = 0.0;
    for (int x = 0; x < n; ++x)
        if (!p->occ[x]) s += R[a * n + x] * b[x];
    return s;
}

/* Leaf value, Eq. 4 with Gamma = {Q(., a)}: max_a sum_x b(x) Q(a, x).
 * Ties keep the lowest action index.                                      */
double or_leaf_value(const or_problem *p, const double *Q, const double *b, double *qa) {
    int n = p->H * p->W;
    double best = -HUGE_VAL;
    for (int a = 0; a < OR_NUM_ACTIONS; ++a) {
        double s = 0.0;
        for (int x = 0; x < n; ++x)
            if (!p->occ[x]) s += b[x] * Q[a * n + x];
        if (qa) qa[a] = s;
        if (s > best) best = s;
    }
    return best;
}

/* Philox4x32-10, from Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
 * multiplies with a Weyl-sequence key schedule.                          */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Sample stream of one (V-node, action): counter {k/4, episode, path_lo,
 * (level << 24) | path_hi}, key = seed; word k%4 -> u = (2 (r >> 9) + 1) 2^-24,
 * which is exact in FP32 and lies in (0, 1).                              */
float or_uniform(uint64_t seed, uint32_t episode, int level, uint64_t path, int k) {
    uint32_t ctr[4] = {(uint32_t)(k / 4), episode, (uint32_t)(path & 0xFFFFFFFFu),
                       ((uint32_t)level << 24) | (uint32_t)(path >> 32)};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    uint32_t r = out[k % 4];
    return (float)(2u * (r >> 9) + 1u) * (1.0f / 16777216.0f);
}

/* Forward sampling (Alg. 4) draws z from P(z | b, a); here by inverting the
 * cumulative sum of the exact marginal, in FP32.                          */
int or_sample_obs(const double *P, int nz, float u) {
    float *C = (float *)malloc(sizeof(float) * nz);
    float s = 0.0f;
    for (int z = 0; z < nz; ++z) { s = s + (float)P[z]; C[z] = s; }
    float t = u * C[nz - 1];
    int pick = nz - 1;
    for (int z = 0; z < nz; ++z)
        if (t < C[z]) { pick = z; break; }
    free(C);
    return pick;
}

int or_is_boundary(const double *P, int nz, float u) {
    double tot = 0.0;
    for (int z = 0; z < nz; ++z) tot += P[z];
    double s = 0.0;
    for (int z = 0; z + 1 < nz; ++z) {
        s += P[z];
        if (fabs((double)u - s / tot) < 1e-6) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tree search: Alg. 2 (V-node expansion over every action), Alg. 3 (Q-node:
 * n forward samples, the unique measurements with their frequencies, one
 * belief update and one V-node per unique measurement), Alg. 5 (a leaf's
 * value from the offline bound), Alg. 6 and 7 (Q- and V-node updates).
 * Readings: every V-node above depth d is expanded (full width, level by
 * level); the Q update discounts the children by gamma as Eq. 2 does; the
 * weight of a child is its sample frequency f/K (FREQ) or its marginal
 * P(z)/sum over the sampled z (MARGINAL).                                   */
int or_tree_plan(const or_problem *p, const double *Q, const double *b0,
                 int depth, int K, uint64_t seed, uint32_t episode, int weight_mode,
                 const int *replay, const long *off, int store_levels,
                 int *n_level, int *parent, int *action, int *obs,
                 double *weight, double *pz, double *value,
                 double *R, double *UQ, int *samples, unsigned char *boundary,
                 double *belief, int *root_action, double *root_value,
                 double *root_q, long *boundary_count) {
    const int n = p->H * p->W, nz = p->B + 1, A = OR_NUM_ACTIONS;
    int *label = (int *)malloc(sizeof(int) * n);
    double *Rt = (double *)malloc(sizeof(double) * A * n);
    or_labels(p, label);
    or_reward_table(p, Rt);

    /* beliefs of the current and next level; path codes for the sampler */
    double **lev_b = (double **)calloc(depth + 1, sizeof(double *));
    uint64_t **code = (uint64_t **)calloc(depth + 1, sizeof(uint64_t *));
    long bcount = 0;
    int status = 0;

    /* root V-node */
    n_level[0] = 1;
    lev_b[0] = (double *)malloc(sizeof(double) * n);
    for (int x = 0; x < n; ++x) lev_b[0][x] = p->occ[x] ? 0.0 : b0[x];
    code[0] = (uint64_t *)malloc(sizeof(uint64_t));
    code[0][0] = 0;
    parent[off[0]] = -1; action[off[0]] = -1; obs[off[0]] = -1;
    weight[off[0]] = 1.0; pz[off[0]] = 1.0;

    for (int l = 0; l < depth && status == 0; ++l) {
        const int nl = n_level[l];
        const long base = off[l];
        /* per (node, action): unique sampled measurements and frequencies */
        int *uz = (int *)malloc(sizeof(int) * (size_t)nl * A * K);
        int *uf = (int *)malloc(sizeof(int) * (size_t)nl * A * K);
        double *up = (double *)malloc(sizeof(double) * (size_t)nl * A * K);
        int *un = (int *)calloc((size_t)nl * A, sizeof(int));
        long lb = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : lb)
        for (int i = 0; i < nl; ++i) {
            const double *b = lev_b[l] + (size_t)i * n;
            double *bbar = (double *)malloc(sizeof(double) * n);
            double *P = (double *)malloc(sizeof(double) * nz);
            int *cnt = (int *)malloc(sizeof(int) * nz);
            for (int a = 0; a < A; ++a) {
                const long s = (base + i) * A + a;
                R[s] = or_belief_reward(p, Rt, b, a);
                or_predict(p, b, a, bbar);
                or_obs_marginal(p, label, bbar, P);
                const uint64_t path = code[l][i] * A + (uint64_t)a;
                for (int z = 0; z < nz; ++z) cnt[z] = 0;
                for (int k = 0; k < K; ++k) {
                    float u = or_uniform(seed, episode, l, path, k);
                    int z = replay ? replay[s * K + k] : or_sample_obs(P, nz, u);
                    unsigned char bd = (unsigned char)or_is_boundary(P, nz, u);
                    samples[s * K + k] = z;
                    boundary[s * K + k] = bd;
                    lb += bd;
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
            }
            free(bbar); free(P); free(cnt);
        }
        bcount += lb;
        /* children of level l+1 in (parent, action, z) order */
        long nn = 0;
        for (long s = 0; s < (long)nl * A; ++s) nn += un[s];
        if (off[l] + nl > off[l + 1] || off[l + 1] + nn > off[l + 2]) status = -1;
        if (status == 0) {
            n_level[l + 1] = (int)nn;
            long c = 0;
            for (int i = 0; i < nl; ++i)
                for (int a = 0; a < A; ++a) {
                    const int m = un[(size_t)i * A + a];
                    double psum = 0.0;
                    for (int j = 0; j < m; ++j) psum += up[((size_t)i * A + a) * K + j];
                    for (int j = 0; j < m; ++j) {
                        const long t = off[l + 1] + c + j;
                        parent[t] = i;
                        action[t] = a;
                        obs[t] = uz[((size_t)i * A + a) * K + j];
                        pz[t] = up[((size_t)i * A + a) * K + j];
                        weight[t] = weight_mode == OR_WEIGHT_MARGINAL
                                        ? pz[t] / psum
                                        : (double)uf[((size_t)i * A + a) * K + j] / (double)K;
                    }
                    c += m;
                }
            code[l + 1] = (uint64_t *)malloc(sizeof(uint64_t) * (nn > 0 ? nn : 1));
            const int leaf = (l + 1 == depth);
            if (!leaf || store_levels >= l + 1)
                lev_b[l + 1] = (double *)malloc(sizeof(double) * (size_t)(nn > 0 ? nn : 1) * n);
#pragma omp parallel for schedule(dynamic)
            for (long j = 0; j < nn; ++j) {
                const long t = off[l + 1] + j;
                const double *b = lev_b[l] + (size_t)parent[t] * n;
                code[l + 1][j] = (code[l][parent[t]] * A + (uint64_t)action[t]) * (uint64_t)nz
                                 + (uint64_t)obs[t];
                double *bbar = (double *)malloc(sizeof(double) * n);
                double *bn = lev_b[l + 1] ? lev_b[l + 1] + (size_t)j * n
                                          : (double *)malloc(sizeof(double) * n);
                or_predict(p, b, action[t], bbar);
                or_correct(p, label, bbar, obs[t], bn);           /* Eq. 3 */
                if (leaf) value[t] = or_leaf_value(p, Q, bn, NULL); /* Alg. 5 */
                if (!lev_b[l + 1]) free(bn);
                free(bbar);
            }
        }
        free(uz); free(uf); free(up); free(un);
    }
    if (depth == 0) value[off[0]] = or_leaf_value(p, Q, lev_b[0], NULL);

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
                double uq = R[(off[l] + i) * A + a] + p->gamma * s;
                UQ[(off[l] + i) * A + a] = uq;
                if (uq > best) best = uq;
            }
            value[off[l] + i] = best;
        }
    }
    if (status == 0) {
        int best = 0;
        if (depth == 0) {
            double qa[5];
            *root_value = or_leaf_value(p, Q, lev_b[0], qa);
            for (int a = 0; a < A; ++a) root_q[a] = qa[a];
            for (int a = 1; a < A; ++a) if (qa[a] > qa[best]) best = a;
        } else {
            for (int a = 0; a < A; ++a) root_q[a] = UQ[off[0] * A + a];
            for (int a = 1; a < A; ++a) if (root_q[a] > root_q[best]) best = a;
            *root_value = value[off[0]];
        }
        *root_action = best;
        *boundary_count = bcount;
    }
    if (belief && status == 0)
        for (int l = 0; l <= depth && l <= store_levels; ++l)
            if (lev_b[l])
                memcpy(belief + (size_t)off[l] * n, lev_b[l], sizeof(double) * (size_t)n_level[l] * n);
    for (int l = 0; l <= depth; ++l) { free(lev_b[l]); free(code[l]); }
    free(lev_b); free(code); free(label); free(Rt);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode (adjoint) of the root value.  The plan's value is a function
 * of the slip eps (through T, Sec. II and Eq. 10), the sensor accuracy alpha
 * (through O) and the cost map c (through r and so R and Q).  Everything the
 * forward pass decided is held fixed: the sampled measurements, the FREQ
 * weights f/K, every max over actions (Alg. 7, Eq. 4 over the leaf's
 * alpha-vectors, the Bellman max of each sweep), ties to the lowest index.
 * Only the FREQ weighting is handled: its weights do not depend on the
 * parameters.                                                               */

/* d T(x, a, y) / d eps on the targets of or_transition_row: the intended
 * move (weight 1 - 2 eps) gives -2, each perpendicular slip (eps) gives +1;
 * Eq. 10 folds blocked moves onto x exactly as in the forward row.  Rows of
 * absorbing cells and of the stay action do not depend on eps.             */
int or_transition_row_dslip(const or_problem *p, int x, int a, int *y, double *dpr) {
    int n = 0;
    if (p->occ[x] || x == p->goal || a == 4) {
        y[0] = x; dpr[0] = 0.0;
        return 1;
    }
    int r = x / p->W, c = x % p->W;
    int dirs[3] = {a, (a + 1) % 4, (a + 3) % 4};
    double w[3] = {-2.0, 1.0, 1.0};
    for (int i = 0; i < 3; ++i) {
        int rr = r + DR[dirs[i]], cc = c + DC[dirs[i]];
        int t = is_free(p, rr, cc) ? rr * p->W + cc : x;
        int j;
        for (j = 0; j < n; ++j)
            if (y[j] == t) { dpr[j] += w[i]; break; }
        if (j == n) { y[n] = t; dpr[n] = w[i]; ++n; }
    }
    return n;
}

/* d O(x', z) / d alpha: 1 on the cell's own label, -1/B elsewhere.         */
static double obs_lik_dacc(const or_problem *p, const int *label, int x, int z) {
    return label[x] == z ? 1.0 : -1.0 / (double)p->B;
}

static int argmax5(const double *q) {
    int best = 0;
    for (int a = 1; a < OR_NUM_ACTIONS; ++a)
        if (q[a] > q[best]) best = a;
    return best;
}

int or_tree_backward(const or_problem *p, const double *Q, int depth, int K, const long *off,
                     const int *n_level, const int *parent, const int *action, const int *obs,
                     const double *weight, const double *UQ, const double *belief, double dL_dV,
                     double *Qbar, double *Rbar, double *dslip, double *dacc, double *db0) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS;
    (void)K;
    double qa[OR_NUM_ACTIONS];
    if (depth == 0) {
        /* the root is the leaf: U_V(b0) = max_a sum_x b0(x) Q(a, x) (Eq. 4) */
        const double *b = belief;
        or_leaf_value(p, Q, b, qa);
        const int ap = argmax5(qa);
        for (int x = 0; x < n; ++x) {
            if (p->occ[x]) continue;
            Qbar[ap * n + x] += dL_dV * b[x];
            if (db0) db0[x] += dL_dV * Q[ap * n + x];
        }
        return 0;
    }
    int *label = (int *)malloc(sizeof(int) * n);
    double *Rt = (double *)malloc(sizeof(double) * A * n);
    or_labels(p, label);
    or_reward_table(p, Rt);
    /* adjoint of every V-node's value, top down: Alg. 7 passes it to the
     * chosen action only, Alg. 6 to that action's children times gamma f/K */
    double *u = (double *)calloc((size_t)off[depth + 1], sizeof(double));
    int *best = (int *)calloc((size_t)off[depth + 1], sizeof(int));
    u[off[0]] = dL_dV;
    for (int l = 0; l < depth; ++l) {
        for (int i = 0; i < n_level[l]; ++i) best[off[l] + i] = argmax5(UQ + (off[l] + i) * A);
        for (int j = 0; j < n_level[l + 1]; ++j) {
            const long t = off[l + 1] + j;
            const long pi = off[l] + parent[t];
            if (action[t] == best[pi]) u[t] = p->gamma * weight[t] * u[pi];
        }
    }
    /* adjoint of the belief of every V-node of the level below */
    double *beta_below = NULL;
    double *bbar = (double *)malloc(sizeof(double) * n);
    double *bc = (double *)malloc(sizeof(double) * n);
    double *betac = (double *)malloc(sizeof(double) * n);
    double *g = (double *)malloc(sizeof(double) * n);
    for (int l = depth - 1; l >= 0; --l) {
        double *beta = (double *)calloc((size_t)(n_level[l] > 0 ? n_level[l] : 1) * n, sizeof(double));
        for (int i = 0; i < n_level[l]; ++i) {
            const long si = off[l] + i;
            const double ui = u[si];
            if (ui == 0.0) continue;
            const double *b = belief + (size_t)si * n;
            const int a = best[si];
            or_predict(p, b, a, bbar);                     /* Eq. 3 numerator */
            for (int y = 0; y < n; ++y) g[y] = 0.0;
            for (int j = 0; j < n_level[l + 1]; ++j) {
                const long t = off[l + 1] + j;
                if (parent[t] != i || action[t] != a) continue;
                const int z = obs[t];
                const double P = or_correct(p, label, bbar, z, bc);   /* Eq. 3 */
                if (l + 1 == depth) {
                    /* leaf: V(b') = sum_y b'(y) Q(a', y) with a' its argmax */
                    or_leaf_value(p, Q, bc, qa);
                    const int ap = argmax5(qa);
                    for (int y = 0; y < n; ++y) {
                        betac[y] = p->occ[y] ? 0.0 : u[t] * Q[ap * n + y];
                        if (!p->occ[y]) Qbar[ap * n + y] += u[t] * bc[y];
                    }
                } else {
                    memcpy(betac, beta_below + (size_t)j * n, sizeof(double) * n);
                }
                /* b' = O_z bbar / P(z):  dL/dbbar = O_z (beta' - <beta', b'>) / P,
                 * dL/dO_z(y) = bbar(y) (beta'(y) - <beta', b'>) / P           */
                double s = 0.0;
                for (int y = 0; y < n; ++y) s += betac[y] * bc[y];
                for (int y = 0; y < n; ++y) {
                    const double d = (betac[y] - s) / P;
                    g[y] += or_obs_lik(p, label, y, z) * d;
                    *dacc += bbar[y] * d * obs_lik_dacc(p, label, y, z);
                }
            }
            /* U_Q(b, a) = R(b, a) + ...:  R(b, a) = sum_x R(x, a) b(x), and
             * bbar = T_a^T b:  dL/db(x) = u R(x, a) + sum_y T(x, a, y) g(y) */
            double *bi = beta + (size_t)i * n;
            for (int x = 0; x < n; ++x) {
                if (p->occ[x]) continue;
                int ys[3]; double pr[3];
                int m = or_transition_row(p, x, a, ys, pr);
                double s = 0.0;
                for (int k = 0; k < m; ++k) s += pr[k] * g[ys[k]];
                bi[x] = ui * Rt[a * n + x] + s;
                Rbar[a * n + x] += ui * b[x];
                m = or_transition_row_dslip(p, x, a, ys, pr);
                double ds = 0.0;
                for (int k = 0; k < m; ++k) ds += pr[k] * g[ys[k]];
                *dslip += b[x] * ds;
            }
        }
        free(beta_below);
        beta_below = beta;
    }
    if (db0)
        for (int x = 0; x < n; ++x) db0[x] += beta_below[x];
    free(beta_below); free(bbar); free(bc); free(betac); free(g);
    free(u); free(best); free(label); free(Rt);
    return 0;
}

int or_vi_backward(const or_problem *p, int sweeps, const double *Qbar, double *Rbar,
                   double *dslip, double *dcost) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS;
    double *R = (double *)malloc(sizeof(double) * A * n);
    double *V = (double *)calloc((size_t)(sweeps + 1) * n, sizeof(double));  /* V_0 .. V_S */
    int *astar = (int *)malloc(sizeof(int) * (size_t)(sweeps > 0 ? sweeps : 1) * n);
    or_reward_table(p, R);
    /* the forward sweeps of or_value_iteration, every V_k and argmax kept */
    for (int k = 0; k < sweeps; ++k) {
        const double *Vk = V + (size_t)k * n;
        double *Vn = V + (size_t)(k + 1) * n;
        for (int x = 0; x < n; ++x) {
            astar[(size_t)k * n + x] = -1;
            if (p->occ[x] || x == p->goal) { Vn[x] = 0.0; continue; }
            double best = -HUGE_VAL;
            for (int a = 0; a < A; ++a) {
                int y[3]; double pr[3];
                int m = or_transition_row(p, x, a, y, pr);
                double s = 0.0;
                for (int j = 0; j < m; ++j) s += pr[j] * Vk[y[j]];
                double q = R[a * n + x] + p->gamma * s;
                if (q > best) { best = q; astar[(size_t)k * n + x] = a; }
            }
            Vn[x] = best;
        }
    }
    double *lam = (double *)calloc(n, sizeof(double));
    double *lam_prev = (double *)calloc(n, sizeof(double));
    /* Q(a, x) = R(x, a) + gamma sum_y T(x, a, y) V_S(y) */
    const double *VS = V + (size_t)sweeps * n;
    for (int x = 0; x < n; ++x) {
        if (p->occ[x] || x == p->goal) continue;
        for (int a = 0; a < A; ++a) {
            const double qb = Qbar[a * n + x];
            if (qb == 0.0) continue;
            Rbar[a * n + x] += qb;
            int y[3]; double pr[3];
            int m = or_transition_row(p, x, a, y, pr);
            for (int j = 0; j < m; ++j) lam[y[j]] += p->gamma * qb * pr[j];
            m = or_transition_row_dslip(p, x, a, y, pr);
            for (int j = 0; j < m; ++j) *dslip += p->gamma * qb * pr[j] * VS[y[j]];
        }
    }
    /* V_{k+1}(x) = R(x, a*) + gamma sum_y T(x, a*, y) V_k(y), k = S-1 .. 0 */
    for (int k = sweeps - 1; k >= 0; --k) {
        const double *Vk = V + (size_t)k * n;
        for (int y = 0; y < n; ++y) lam_prev[y] = 0.0;
        for (int x = 0; x < n; ++x) {
            if (p->occ[x] || x == p->goal) continue;
            const double lx = lam[x];
            if (lx == 0.0) continue;
            const int a = astar[(size_t)k * n + x];
            Rbar[a * n + x] += lx;
            int y[3]; double pr[3];
            int m = or_transition_row(p, x, a, y, pr);
            for (int j = 0; j < m; ++j) lam_prev[y[j]] += p->gamma * lx * pr[j];
            m = or_transition_row_dslip(p, x, a, y, pr);
            for (int j = 0; j < m; ++j) *dslip += p->gamma * lx * pr[j] * Vk[y[j]];
        }
        double *t = lam; lam = lam_prev; lam_prev = t;
    }
    /* R(x, a) = sum_y T(x, a, y) r(y), r(y) = -1 - c(y) off the goal */
    for (int x = 0; x < n; ++x) {
        if (p->occ[x] || x == p->goal) continue;
        for (int a = 0; a < A; ++a) {
            const double rb = Rbar[a * n + x];
            if (rb == 0.0) continue;
            int y[3]; double pr[3];
            int m = or_transition_row_dslip(p, x, a, y, pr);
            for (int j = 0; j < m; ++j) *dslip += rb * pr[j] * stage_reward(p, y[j]);
            m = or_transition_row(p, x, a, y, pr);
            for (int j = 0; j < m; ++j)
                if (y[j] != p->goal && dcost) dcost[y[j]] -= rb * pr[j];
        }
    }
    free(R); free(V); free(astar); free(lam); free(lam_prev);
    return 0;
}

/* ---- Fast Informed Bound (Sec. IV-A) ---------------------------------- */

/* One application of the FIB alpha-vector Bellman operator, Eq. 7:
 *   alpha'^a(x) = R(x, a) + gamma sum_z max_a' sum_x' O(x', z) T(x, a, x') alpha^a'(x')
 * for every free, non-goal cell x and action a; the sum over x' runs over
 * the support of T(x, a, .) (every other term is zero) and z over all B + 1
 * observations.  The goal and occupied cells keep alpha = 0, as V does in
 * the value iteration (absorbing, nothing earned there).  alpha, out: [5*n],
 * action-major.  Returns max |out - alpha| over every (a, x).              */
double or_fib_sweep(const or_problem *p, const int *label, const double *R, const double *alpha,
                    double *out) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS, nz = p->B + 1;
    double res = 0.0;
#pragma omp parallel for schedule(static) reduction(max : res)
    for (int x = 0; x < n; ++x) {
        for (int a = 0; a < A; ++a) {
            double v = 0.0;
            if (!p->occ[x] && x != p->goal) {
                int y[3]; double pr[3];
                const int m = or_transition_row(p, x, a, y, pr);
                double sz = 0.0;
                for (int z = 0; z < nz; ++z) {
                    double best = -HUGE_VAL;
                    for (int b = 0; b < A; ++b) {
                        double s = 0.0;
                        for (int j = 0; j < m; ++j)
                            s += or_obs_lik(p, label, y[j], z) * pr[j] * alpha[b * n + y[j]];
                        if (s > best) best = s;
                    }
                    sz += best;
                }
                v = R[a * n + x] + p->gamma * sz;
            }
            out[a * n + x] = v;
            const double d = fabs(v - alpha[a * n + x]);
            if (d > res) res = d;
        }
    }
    return res;
}

/* FIB value iteration (Sec. IV-A: Eq. 7 is a monotone contraction, so Jacobi
 * sweeps converge): alpha_0 = 0, alpha_{k+1} = Eq. 7 applied to alpha_k;
 * stops at the first sweep whose max-abs change is below tol, or after
 * exactly `truncated` sweeps when truncated > 0.  Returns 0, or 1 when
 * max_sweeps ran out first.  alpha: [5*n]; residual_hist nullable.        */
int or_fib_iteration(const or_problem *p, double tol, int max_sweeps, int truncated, double *alpha,
                     int *sweeps, double *residual, double *residual_hist) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS;
    int *label = (int *)malloc(sizeof(int) * n);
    double *R = (double *)malloc(sizeof(double) * A * n);
    double *next = (double *)malloc(sizeof(double) * A * n);
    or_labels(p, label);
    or_reward_table(p, R);
    for (int i = 0; i < A * n; ++i) alpha[i] = 0.0;
    const int limit = truncated > 0 ? truncated : max_sweeps;
    int k = 0, status = 1;
    double res = 0.0;
    while (k < limit) {
        res = or_fib_sweep(p, label, R, alpha, next);
        memcpy(alpha, next, sizeof(double) * A * n);
        if (residual_hist) residual_hist[k] = res;
        ++k;
        if (truncated <= 0 && res < tol) { status = 0; break; }
    }
    if (truncated > 0) status = 0;
    *sweeps = k;
    *residual = res;
    free(label); free(R); free(next);
    return status;
}

/* ---- Point-based value iteration (Sec. IV-B) --------------------------- */

/* Pessimistic start of the PBVI alpha-vectors: every policy earns at least
 * R_min = min over free, non-goal x and a of R(x, a) per step, so
 * alpha_0 = R_min / (1 - gamma) on those cells (0 on the goal and occupied
 * cells) is below V* everywhere.  alpha0: [n].                            */
void or_pbvi_init(const or_problem *p, double *alpha0) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS;
    double *R = (double *)malloc(sizeof(double) * A * n);
    or_reward_table(p, R);
    double rmin = HUGE_VAL;
    for (int x = 0; x < n; ++x) {
        if (p->occ[x] || x == p->goal) continue;
        for (int a = 0; a < A; ++a)
            if (R[a * n + x] < rmin) rmin = R[a * n + x];
    }
    for (int x = 0; x < n; ++x) alpha0[x] = (p->occ[x] || x == p->goal) ? 0.0 : rmin / (1.0 - p->gamma);
    free(R);
}

/* Belief set expansion (Sec. IV-B): every point b_j of the set yields one
 * new point by forward sampling one action-observation step from it: the
 * action uniformly, a = floor(5 u_a), then z ~ P(z | b_j, a) by the inverse
 * CDF of Alg. 3-4's reading, then b' = tau(b_j, a, z) (Eq. 3).  The uniforms
 * are the Philox stream of the tree search with level code 255 (never a tree
 * level), episode word = the expansion round, path = j: u_a is its word 0,
 * u_z its word 1.  B: [nB][n]; out: [nB][n]; action, obs, boundary: [nB].  */
int or_pbvi_expand(const or_problem *p, const double *B, int nB, int round, uint64_t seed, double *out,
                   int *action, int *obs, int *boundary) {
    const int n = p->H * p->W, nz = p->B + 1;
    int *label = (int *)malloc(sizeof(int) * n);
    or_labels(p, label);
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nB; ++j) {
        double *bbar = (double *)malloc(sizeof(double) * n);
        double *P = (double *)malloc(sizeof(double) * nz);
        const float ua = or_uniform(seed, (uint32_t)round, 255, (uint64_t)j, 0);
        int a = (int)floor((double)ua * 5.0);
        if (a > 4) a = 4;
        or_predict(p, B + (size_t)j * n, a, bbar);
        or_obs_marginal(p, label, bbar, P);
        const float uz = or_uniform(seed, (uint32_t)round, 255, (uint64_t)j, 1);
        const int z = or_sample_obs(P, nz, uz);
        or_correct(p, label, bbar, z, out + (size_t)j * n);
        action[j] = a;
        obs[j] = z;
        boundary[j] = or_is_boundary(P, nz, uz);
        free(bbar); free(P);
    }
    free(label);
    return 0;
}

/* Eq. 8's argmax: the first index attaining the largest value (exact ties
 * to the lowest index).                                                    */
static int pbvi_pick(const double *v, int n) {
    int best = 0;
    for (int i = 1; i < n; ++i)
        if (v[i] > v[best]) best = i;
    return best;
}

/* One PBVI alpha-vector backup, Eq. 8, at every point b of B given the set
 * Gamma (nG vectors of n values):
 *   for each action a and observation z, the vector of Gamma maximising
 *     sum_x sum_x' O(x', z) T(x, a, x') alpha(x') b(x)          (ties: pbvi_pick),
 *   Q_b(a) = R(b, a) + gamma sum_z (that vector's sum),
 *   a*(b) = argmax_a Q_b(a)                                      (ties: pbvi_pick),
 * and the new vector of b is
 *   alpha_b(x) = R(x, a*) + gamma sum_z sum_x' O(x', z) T(x, a*, x') alpha_{i*(z)}(x')
 * on free, non-goal x, 0 on the goal and occupied cells (their value is 0
 * under every policy).  Gout: [nB][n]; value[b] = Q_b(a*) = sum_x b(x) alpha_b(x);
 * astar[b]; best: [nB][nz] the maximising indices for a*; q: [nB][5]
 * (nullable) every Q_b(a); score: [nB][5][nz][nG] (nullable) every sum.   */
int or_pbvi_backup(const or_problem *p, const double *B, int nB, const double *G, int nG, double *Gout,
                   double *value, int *astar, int *best, double *q, double *score) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS, nz = p->B + 1;
    int *label = (int *)malloc(sizeof(int) * n);
    double *R = (double *)malloc(sizeof(double) * A * n);
    or_labels(p, label);
    or_reward_table(p, R);
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < nB; ++j) {
        const double *b = B + (size_t)j * n;
        int *bi = (int *)malloc(sizeof(int) * A * nz);
        double *sc = (double *)malloc(sizeof(double) * (nG > 0 ? nG : 1));
        double qa[OR_NUM_ACTIONS];
        for (int a = 0; a < A; ++a) {
            double qv = 0.0;
            for (int x = 0; x < n; ++x) qv += R[a * n + x] * b[x];   /* R(b, a) */
            for (int z = 0; z < nz; ++z) {
                for (int i = 0; i < nG; ++i) {
                    const double *al = G + (size_t)i * n;
                    double s = 0.0;
                    for (int x = 0; x < n; ++x) {
                        if (b[x] == 0.0) continue;
                        int y[3]; double pr[3];
                        const int m = or_transition_row(p, x, a, y, pr);
                        for (int t = 0; t < m; ++t)
                            s += or_obs_lik(p, label, y[t], z) * pr[t] * al[y[t]] * b[x];
                    }
                    if (score) score[(((size_t)j * A + a) * nz + z) * nG + i] = s;
                    sc[i] = s;
                }
                const int arg = pbvi_pick(sc, nG);
                bi[a * nz + z] = arg;
                qv += p->gamma * sc[arg];
            }
            qa[a] = qv;
            if (q) q[(size_t)j * A + a] = qv;
        }
        const int as = pbvi_pick(qa, A);
        astar[j] = as;
        value[j] = qa[as];
        for (int z = 0; z < nz; ++z) best[(size_t)j * nz + z] = bi[as * nz + z];
        double *out = Gout + (size_t)j * n;
        for (int x = 0; x < n; ++x) {
            if (p->occ[x] || x == p->goal) { out[x] = 0.0; continue; }
            int y[3]; double pr[3];
            const int m = or_transition_row(p, x, as, y, pr);
            double s = 0.0;
            for (int z = 0; z < nz; ++z) {
                const double *al = G + (size_t)bi[as * nz + z] * n;
                for (int t = 0; t < m; ++t) s += or_obs_lik(p, label, y[t], z) * pr[t] * al[y[t]];
            }
            out[x] = R[as * n + x] + p->gamma * s;
        }
        free(bi); free(sc);
    }
    free(label); free(R);
    return 0;
}

/* ---- AEMS bookkeeping over a tree (Alg. 5-7, Eq. 9) --------------------- */

/* Lower bounds, heuristics and the V-node to expand, bottom-up over the
 * flat arrays of an or_tree_plan tree (level l at [off[l], off[l] + n_level[l]),
 * children ordered by (parent, action, z)).  Leaves (level depth, Alg. 5):
 * L_V = Lleaf[j] (V_PBVI of the leaf belief), H_V = U_V - L_V, E_V = the
 * leaf itself (its index within the leaf level).  Q-node (Alg. 6, discounted
 * like U_Q): L_Q = R + gamma sum_children weight L_V; the child maximising
 * gamma weight H_V (ties: the first in order) gives H_Q = gamma weight H_V
 * and E_Q = its E_V.  V-node (Alg. 7 with Eq. 9's H(b, a) = 1 for the action
 * maximising U_Q, ties to the lowest): L_V = max_a L_Q, H_V = H_Q and
 * E_V = E_Q of that action.  A Q-node without children keeps L_Q = R,
 * H_Q = 0, E_Q = -1.  Outputs: LV, HV, EV [tot]; LQ, HQ, EQ [tot * 5]
 * (internal nodes).                                                       */
int or_tree_bounds(int depth, const long *off, const int *n_level, const int *parent, const int *action,
                   const double *weight, const double *R, const double *UQ, const double *value,
                   const double *Lleaf, double gamma, double *LV, double *HV, int *EV, double *LQ,
                   double *HQ, int *EQ) {
    const int A = OR_NUM_ACTIONS;
    const long s = off[depth];
    for (int j = 0; j < n_level[depth]; ++j) {
        LV[s + j] = Lleaf[j];
        HV[s + j] = value[s + j] - Lleaf[j];
        EV[s + j] = j;
    }
    for (int l = depth - 1; l >= 0; --l) {
        const long sl = off[l], sc = off[l + 1];
        const int n = n_level[l], nc = n_level[l + 1];
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < A; ++a) {
                const long q = (sl + i) * A + a;
                LQ[q] = R[q];
                HQ[q] = 0.0;
                EQ[q] = -1;
            }
        double *sum = (double *)calloc((size_t)n * A, sizeof(double));
        int *have = (int *)calloc((size_t)n * A, sizeof(int));
        for (int j = 0; j < nc; ++j) {
            const int i = parent[sc + j], a = action[sc + j];
            const long q = (sl + i) * A + a;
            const double w = weight[sc + j];
            sum[(long)i * A + a] += w * LV[sc + j];
            const double h = gamma * w * HV[sc + j];
            if (!have[(long)i * A + a] || h > HQ[q]) {
                HQ[q] = h;
                EQ[q] = EV[sc + j];
                have[(long)i * A + a] = 1;
            }
        }
        for (int i = 0; i < n; ++i) {
            double lmax = -HUGE_VAL;
            int au = 0;
            for (int a = 0; a < A; ++a) {
                const long q = (sl + i) * A + a;
                if (have[(long)i * A + a]) LQ[q] = R[q] + gamma * sum[(long)i * A + a];
                if (LQ[q] > lmax) lmax = LQ[q];
                if (UQ[q] > UQ[(sl + i) * A + au]) au = a;
            }
            LV[sl + i] = lmax;
            HV[sl + i] = HQ[(sl + i) * A + au];
            EV[sl + i] = EQ[(sl + i) * A + au];
        }
        free(sum); free(have);
    }
    return 0;
}

/* ---- Best-first QV-Tree Search (Alg. 1 inner loop, Alg. 2-7, Eq. 9) ----- */

/* Recompute Q-node (v, a) from its children (Alg. 6) and V-node v from its
 * Q-nodes (Alg. 7 with Eq. 9's H(b, a)); the same rules as or_tree_bounds. */
static void bf_update_node(int v, double gamma, const int *cbeg, const int *ccnt, const double *Rq,
                           const double *w, double *U, double *L, double *Hh, int *E, double *UQ, double *LQ,
                           double *HQ, int *EQ) {
    const int A = OR_NUM_ACTIONS;
    for (int a = 0; a < A; ++a) {
        const int q = v * A + a;
        double su = 0.0, sl = 0.0, bh = 0.0;
        int be = -1;
        for (int c = cbeg[q]; c < cbeg[q] + ccnt[q]; ++c) {
            su += w[c] * U[c];
            sl += w[c] * L[c];
            const double h = gamma * w[c] * Hh[c];
            if (be < 0 || h > bh) { bh = h; be = E[c]; }
        }
        UQ[q] = Rq[q] + gamma * su;
        LQ[q] = Rq[q] + gamma * sl;
        HQ[q] = bh;
        EQ[q] = be;
    }
    int au = 0;
    double lmax = LQ[v * A];
    for (int a = 1; a < A; ++a) {
        if (UQ[v * A + a] > UQ[v * A + au]) au = a;
        if (LQ[v * A + a] > lmax) lmax = LQ[v * A + a];
    }
    U[v] = UQ[v * A + au];
    L[v] = lmax;
    Hh[v] = HQ[v * A + au];
    E[v] = EQ[v * A + au];
}

/* The smallest gap among the comparisons that point the root's E at the
 * node to expand, following them down from the root: at every expanded
 * V-node, the largest U_Q against each other action's (Alg. 7 and Eq. 9
 * follow the action maximising U_Q), and among the children of that
 * Q-node the largest gamma * weight * H_V against each other child's
 * (Alg. 6).  HUGE_VAL when the root is still a leaf.                        */
static double bf_margin(double gamma, const int *cbeg, const int *ccnt, const double *UQ, const double *w,
                        const double *Hh) {
    const int A = OR_NUM_ACTIONS;
    double m = HUGE_VAL;
    int u = 0;
    while (ccnt[u * A] > 0) {
        int au = 0;
        for (int a = 1; a < A; ++a)
            if (UQ[u * A + a] > UQ[u * A + au]) au = a;
        for (int a = 0; a < A; ++a)
            if (a != au && UQ[u * A + au] - UQ[u * A + a] < m) m = UQ[u * A + au] - UQ[u * A + a];
        const int q = u * A + au;
        int cb = -1;
        double bh = 0.0;
        for (int c = cbeg[q]; c < cbeg[q] + ccnt[q]; ++c) {
            const double h = gamma * w[c] * Hh[c];
            if (cb < 0 || h > bh) { bh = h; cb = c; }
        }
        for (int c = cbeg[q]; c < cbeg[q] + ccnt[q]; ++c)
            if (c != cb && bh - gamma * w[c] * Hh[c] < m) m = bh - gamma * w[c] * Hh[c];
        u = cb;
    }
    return m;
}

/* Alg. 1's planning loop: starting from the root V-node of b0 (U = V_U(b0)
 * with the upper-bound alpha-vectors Qu, e.g. FIB; L = V_PBVI(b0) =
 * max_i G_i . b0; H = U - L; E = root), each iteration expands the V-node
 * the root's E points at (Alg. 2: all five actions; Alg. 3: K forward
 * samples of z, the unique ones with frequencies f, children tau(b, a, z)
 * with weight f / K, Alg. 5: U, L, H, E of each child) and updates it and
 * its ancestors (Alg. 6-7).  Node ids are assigned in creation order,
 * children of a Q-node in ascending z.  The samples of (V-node, a) are the
 * Philox stream of the level-synchronous tree: level = depth, path = the
 * node's mixed-radix code * 5 + a.  A node created at max_depth is closed:
 * its H is 0, so the search turns elsewhere.  Planning stops early when the
 * node to expand lies at max_depth (every open gap is 0) or the next
 * expansion could overflow max_nodes.
 * Outputs per node: parent, action, obs, depth, weight, U, L, H, E; per
 * Q-node (v * 5 + a): R, U_Q, L_Q, H_Q, E_Q, first child, children;
 * expanded[it] the node expanded at iteration it (-1 after a stop);
 * *n_nodes; *boundary draws within 1e-6 of a CDF step.  Returns the
 * iterations run.  belief: [max_nodes][n] scratch.  margin (nullable,
 * [iters]): for each iteration, the smallest gap among the comparisons that
 * pointed the root's E at the node it expanded (bf_margin); a comparison
 * whose gap is within rounding can order differently in another precision. */
int or_bestfirst(const or_problem *p, const double *Qu, const double *G, int nG, const double *b0, int K,
                 uint64_t seed, uint32_t episode, int iters, int max_depth, int max_nodes, double *belief,
                 int *n_nodes, int *expanded, int *vparent, int *vaction, int *vobs, int *vdepth, double *vweight,
                 double *U, double *L, double *Hh, int *E, double *Rq, double *UQ, double *LQ, double *HQ, int *EQ,
                 int *cbeg, int *ccnt, long *boundary, double *margin) {
    const int n = p->H * p->W, nz = p->B + 1, A = OR_NUM_ACTIONS;
    int *label = (int *)malloc(sizeof(int) * n);
    double *Rt = (double *)malloc(sizeof(double) * A * n);
    double *bbar = (double *)malloc(sizeof(double) * n);
    double *P = (double *)malloc(sizeof(double) * nz);
    int *cnt = (int *)malloc(sizeof(int) * nz);
    uint64_t *code = (uint64_t *)malloc(sizeof(uint64_t) * max_nodes);
    or_labels(p, label);
    or_reward_table(p, Rt);
    *boundary = 0;
    for (int i = 0; i < max_nodes * A; ++i) { cbeg[i] = 0; ccnt[i] = 0; Rq[i] = UQ[i] = LQ[i] = HQ[i] = 0.0; EQ[i] = -1; }
    /* the root */
    for (int x = 0; x < n; ++x) belief[x] = p->occ[x] ? 0.0 : b0[x];
    vparent[0] = -1; vaction[0] = -1; vobs[0] = -1; vdepth[0] = 0; vweight[0] = 1.0; code[0] = 0;
    U[0] = or_leaf_value(p, Qu, belief, NULL);
    {
        double best = -HUGE_VAL;
        for (int i = 0; i < nG; ++i) {
            double s = 0.0;
            for (int x = 0; x < n; ++x) s += G[(size_t)i * n + x] * belief[x];
            if (s > best) best = s;
        }
        L[0] = best;
    }
    Hh[0] = U[0] - L[0];
    E[0] = 0;
    int nn = 1, it = 0;
    for (; it < iters; ++it) {
        int v = E[0];
        const int room = A * (K < nz ? K : nz);
        if (vdepth[v] >= max_depth || nn + room > max_nodes) break;
        if (margin) margin[it] = bf_margin(p->gamma, cbeg, ccnt, UQ, vweight, Hh);
        const double *b = belief + (size_t)v * n;
        for (int a = 0; a < A; ++a) {
            const int q = v * A + a;
            Rq[q] = or_belief_reward(p, Rt, b, a);
            or_predict(p, b, a, bbar);
            or_obs_marginal(p, label, bbar, P);
            const uint64_t path = code[v] * A + (uint64_t)a;
            for (int z = 0; z < nz; ++z) cnt[z] = 0;
            for (int k = 0; k < K; ++k) {
                const float u = or_uniform(seed, episode, vdepth[v], path, k);
                cnt[or_sample_obs(P, nz, u)] += 1;
                *boundary += or_is_boundary(P, nz, u);
            }
            cbeg[q] = nn;
            for (int z = 0; z < nz; ++z) {
                if (!cnt[z]) continue;
                const int c = nn++;
                double *bc = belief + (size_t)c * n;
                or_correct(p, label, bbar, z, bc);
                vparent[c] = v; vaction[c] = a; vobs[c] = z; vdepth[c] = vdepth[v] + 1;
                vweight[c] = (double)cnt[z] / (double)K;
                code[c] = path * (uint64_t)nz + (uint64_t)z;
                U[c] = or_leaf_value(p, Qu, bc, NULL);
                double best = -HUGE_VAL;
                for (int i = 0; i < nG; ++i) {
                    double s = 0.0;
                    for (int x = 0; x < n; ++x) s += G[(size_t)i * n + x] * bc[x];
                    if (s > best) best = s;
                }
                L[c] = best;
                /* a node at the depth limit is closed: no gap left to draw the search */
                Hh[c] = vdepth[c] < max_depth ? U[c] - L[c] : 0.0;
                E[c] = c;
            }
            ccnt[q] = nn - cbeg[q];
        }
        /* the expanded node, then its ancestors up to the root */
        for (int u = v; u >= 0; u = vparent[u])
            bf_update_node(u, p->gamma, cbeg, ccnt, Rq, vweight, U, L, Hh, E, UQ, LQ, HQ, EQ);
        expanded[it] = v;
    }
    for (int t = it; t < iters; ++t) expanded[t] = -1;
    *n_nodes = nn;
    free(label); free(Rt); free(bbar); free(P); free(cnt); free(code);
    return it;
}

/* ---- Closed-loop episodes (Alg. 1 outer loop, Eq. 1) ------------------- */

/* The true system's step: from x under action a, the motion outcome is
 * drawn with u_m (word 0) and the measurement at the new cell with u_o
 * (word 1) of the Philox stream {0, episode e, path = step, level code 254}.
 * Motion: the intended move if u_m < 1 - 2 eps, the first perpendicular
 * (a + 1) if u_m < 1 - eps, else the second (a + 3), in FP32 as the kernel
 * decides; a blocked move stays (Eq. 10); stay, the goal and occupied
 * cells stay.  Measurement: z from O(x', .) by the inverse CDF of
 * or_sample_obs.                                                            */
int or_env_step(const or_problem *p, const int *label, int x, int a, uint64_t seed, uint32_t e, int step, int *z_out) {
    const float um = or_uniform(seed, e, 254, (uint64_t)step, 0);
    const float uo = or_uniform(seed, e, 254, (uint64_t)step, 1);
    int y = x;
    if (!p->occ[x] && x != p->goal && a != 4) {
        const float eps = (float)p->slip;
        const float fwd = 1.0f - 2.0f * eps;
        const int d = um < fwd ? a : (um < fwd + eps ? (a + 1) % 4 : (a + 3) % 4);
        const int r = x / p->W + DR[d], c = x % p->W + DC[d];
        if (is_free(p, r, c)) y = r * p->W + c;
    }
    const int nz = p->B + 1;
    double *P = (double *)malloc(sizeof(double) * nz);
    for (int z = 0; z < nz; ++z) P[z] = or_obs_lik(p, label, y, z);
    *z_out = or_sample_obs(P, nz, uo);
    free(P);
    return y;
}

/* E episodes of the loop of Alg. 1 (its outer loop): plan from the belief
 * (the level-synchronous tree, Philox episode word = step * E + e), execute
 * the root action on the true state, receive a measurement, update the
 * belief by Eq. 3, until the goal is reached or max_steps.  Inputs b0s
 * [E][n], x0s [E].  Outputs: actions, obs [E][max_steps], states
 * [E][max_steps + 1] (-1 after the end), steps [E] (moves made), success
 * [E] (goal reached), ret [E] (sum of gamma^t r(x_{t+1}), Eq. 1), root_gap
 * [E][max_steps] (the gap between the two best root Q-values, for deciding
 * near-ties), boundary [E][max_steps] (draws near a CDF step in the plan).  */
int or_closed_loop(const or_problem *p, const double *Q, int E, const double *b0s, const int *x0s, int depth, int K,
                   uint64_t seed, int max_steps, int *actions, int *obs, int *states, int *steps, int *success,
                   double *ret, double *root_gap, long *boundary) {
    const int n = p->H * p->W, A = OR_NUM_ACTIONS, nz = p->B + 1;
    int *label = (int *)malloc(sizeof(int) * n);
    or_labels(p, label);
    /* tree capacity (5 min(K, |Z|))^l per level */
    long *off = (long *)malloc(sizeof(long) * (depth + 2));
    off[0] = 0;
    long cap = 1;
    for (int l = 0; l <= depth; ++l) {
        off[l + 1] = off[l] + cap;
        cap *= A * (K < nz ? K : nz);
    }
    const long tot = off[depth + 1];
    int *n_level = (int *)malloc(sizeof(int) * (depth + 1));
    int *par = (int *)malloc(sizeof(int) * tot), *act = (int *)malloc(sizeof(int) * tot);
    int *ob = (int *)malloc(sizeof(int) * tot);
    double *wt = (double *)malloc(sizeof(double) * tot), *pz = (double *)malloc(sizeof(double) * tot);
    double *val = (double *)malloc(sizeof(double) * tot);
    double *R = (double *)malloc(sizeof(double) * tot * A), *UQ = (double *)malloc(sizeof(double) * tot * A);
    int *samp = (int *)malloc(sizeof(int) * tot * A * K);
    unsigned char *bd = (unsigned char *)malloc(tot * A * K);
    double *b = (double *)malloc(sizeof(double) * n), *bbar = (double *)malloc(sizeof(double) * n);
    for (int e = 0; e < E; ++e) {
        for (int x = 0; x < n; ++x) b[x] = b0s[(size_t)e * n + x];
        int x = x0s[e];
        double g = 1.0, rsum = 0.0;
        int t = 0, ok = 0;
        states[(size_t)e * (max_steps + 1)] = x;
        for (; t < max_steps && x != p->goal; ++t) {
            int ra; double rv, rq[OR_NUM_ACTIONS]; long bc = 0;
            or_tree_plan(p, Q, b, depth, K, seed, (uint32_t)(t * E + e), 0, NULL, off, -1, n_level, par, act, ob,
                         wt, pz, val, R, UQ, samp, bd, NULL, &ra, &rv, rq, &bc);
            double q1 = -HUGE_VAL, q2 = -HUGE_VAL;
            for (int a = 0; a < A; ++a) {
                if (rq[a] > q1) { q2 = q1; q1 = rq[a]; }
                else if (rq[a] > q2) q2 = rq[a];
            }
            root_gap[(size_t)e * max_steps + t] = q1 - q2;
            boundary[(size_t)e * max_steps + t] = bc;
            int z;
            const int y = or_env_step(p, label, x, ra, seed, (uint32_t)e, t, &z);
            actions[(size_t)e * max_steps + t] = ra;
            obs[(size_t)e * max_steps + t] = z;
            rsum += g * (y == p->goal ? 100.0 : -1.0 - (p->cost ? p->cost[y] : 0.0));
            g *= p->gamma;
            or_predict(p, b, ra, bbar);
            or_correct(p, label, bbar, z, b);
            x = y;
            states[(size_t)e * (max_steps + 1) + t + 1] = x;
        }
        ok = (x == p->goal);
        for (int s = t; s < max_steps; ++s) {
            actions[(size_t)e * max_steps + s] = -1;
            obs[(size_t)e * max_steps + s] = -1;
            root_gap[(size_t)e * max_steps + s] = 0.0;
            boundary[(size_t)e * max_steps + s] = 0;
            states[(size_t)e * (max_steps + 1) + s + 1] = -1;
        }
        steps[e] = t;
        success[e] = ok;
        ret[e] = rsum;
    }
    free(label); free(off); free(n_level); free(par); free(act); free(ob); free(wt); free(pz); free(val);
    free(R); free(UQ); free(samp); free(bd); free(b); free(bbar);
    return 0;
}

/* ---- Ancestral forward sampling, Alg. 4 as written ---------------------- */

/* K measurement samples for (b, a), each by Alg. 4's three stages: x ~ b
 * (inverse CDF over the cells in index order), x' ~ T(x, a, .) (the
 * system's motion rule of or_env_step), z ~ O(x', .) (or_sample_obs).  The
 * uniforms of sample k are words 3k, 3k + 1, 3k + 2 of the Philox stream of
 * (level, path); the CDF of b runs in FP32, as the sampler kernels' do.    */
void or_forward_sample(const or_problem *p, const double *b, int a, int K, uint64_t seed, uint32_t episode,
                       int level, uint64_t path, int *z, int *boundary) {
    const int n = p->H * p->W, nz = p->B + 1;
    int *label = (int *)malloc(sizeof(int) * n);
    float *C = (float *)malloc(sizeof(float) * n);
    double *P = (double *)malloc(sizeof(double) * nz);
    or_labels(p, label);
    float run = 0.0f;
    for (int x = 0; x < n; ++x) {
        run = run + (p->occ[x] ? 0.0f : (float)b[x]);
        C[x] = run;
    }
    for (int k = 0; k < K; ++k) {
        const float u1 = or_uniform(seed, episode, level, path, 3 * k);
        const float u2 = or_uniform(seed, episode, level, path, 3 * k + 1);
        const float u3 = or_uniform(seed, episode, level, path, 3 * k + 2);
        /* x ~ b */
        const float t = u1 * C[n - 1];
        int x = n - 1;
        for (int i = 0; i < n; ++i)
            if (t < C[i]) { x = i; break; }
        /* a draw within 1e-5 of the total from a step of the cumulative sum:
         * another summation order of the same FP32 sums may pick the
         * neighbouring cell there */
        if (boundary) {
            const double tol = 1e-5 * (double)C[n - 1];
            boundary[k] = fabs((double)t - (double)C[x]) < tol || (x > 0 && fabs((double)t - (double)C[x - 1]) < tol);
        }
        /* x' ~ T(x, a, .) */
        int y = x;
        if (!p->occ[x] && x != p->goal && a != 4) {
            const float eps = (float)p->slip;
            const float fwd = 1.0f - 2.0f * eps;
            const int d = u2 < fwd ? a : (u2 < fwd + eps ? (a + 1) % 4 : (a + 3) % 4);
            const int r = x / p->W + DR[d], c = x % p->W + DC[d];
            if (is_free(p, r, c)) y = r * p->W + c;
        }
        /* z ~ O(x', .) */
        for (int zz = 0; zz < nz; ++zz) P[zz] = or_obs_lik(p, label, y, zz);
        z[k] = or_sample_obs(P, nz, u3);
    }
    free(label); free(C); free(P);
}
