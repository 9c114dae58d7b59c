/*
 * plan_client.c -- a plain C user of the C ABI (test infrastructure): builds
 * a small grid model, runs FP64 value iteration and one tree plan, and
 * prints the root result as one JSON line.  Device memory comes from the
 * CUDA runtime; nothing here uses C++ or Python.
 *
 * Usage: plan_client H W seed
 * The grid, beacons, goal and b0 follow a fixed recipe from (H, W, seed) so
 * that the test can rebuild the same problem on the Python side.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "qvts.h"

#define CHECK_QV(call)                                                              \
    do {                                                                            \
        qv_status st_ = (call);                                                     \
        if (st_ != QV_OK) {                                                         \
            fprintf(stderr, "%s failed: %d %s\n", #call, (int)st_, qv_last_error()); \
            return 1;                                                               \
        }                                                                           \
    } while (0)
#define CHECK_CUDA(call)                                                            \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            fprintf(stderr, "%s failed: %s\n", #call, cudaGetErrorString(e_));      \
            return 1;                                                               \
        }                                                                           \
    } while (0)

/* the recipe: a wall segment in the middle row with a gap, two beacons, the
 * goal in the last row, b0 uniform over a 3x3 block in the first rows */
static void make_problem(int H, int W, unsigned seed, unsigned char *occ, int *beacons, int *goal, float *b0) {
    int r, c, P = QV_PITCH(W);
    memset(occ, 0, (size_t)H * P);
    for (r = 0; r < H; ++r)
        for (c = W; c < P; ++c) occ[r * P + c] = 1;
    for (c = 0; c < W; ++c)
        if (c != (int)(seed % (unsigned)W)) occ[(H / 2) * P + c] = 1;
    beacons[0] = 1 * P + 1;
    beacons[1] = (H - 2) * P + (W - 2);
    *goal = (H - 1) * P + (W / 2);
    memset(b0, 0, sizeof(float) * (size_t)H * P);
    for (r = 0; r < 3; ++r)
        for (c = 0; c < 3; ++c) b0[r * P + c + 1] = 1.0f / 9.0f;
}

int main(int argc, char **argv) {
    int H = argc > 1 ? atoi(argv[1]) : 12;
    int W = argc > 2 ? atoi(argv[2]) : 10;
    unsigned seed = argc > 3 ? (unsigned)atoi(argv[3]) : 3u;
    int P = QV_PITCH(W), N = H * P, goal = 0, i;
    unsigned char *h_occ = (unsigned char *)malloc((size_t)N);
    float *h_b0 = (float *)malloc(sizeof(float) * (size_t)N);
    int h_beacons[2];
    qv_model_t m;
    qv_plan_params_t prm;
    qv_plan_result_t res;
    unsigned char *d_occ;
    int *d_beacons, sweeps = 0;
    uint16_t *d_cell;
    double *d_V, residual = 0.0;
    float *d_Q, *d_b0;
    void *d_ws;
    size_t vi_bytes, plan_bytes;

    make_problem(H, W, seed, h_occ, h_beacons, &goal, h_b0);
    CHECK_CUDA(cudaMalloc((void **)&d_occ, (size_t)N));
    CHECK_CUDA(cudaMalloc((void **)&d_beacons, sizeof(h_beacons)));
    CHECK_CUDA(cudaMalloc((void **)&d_cell, sizeof(uint16_t) * (size_t)N));
    CHECK_CUDA(cudaMalloc((void **)&d_V, sizeof(double) * (size_t)N));
    CHECK_CUDA(cudaMalloc((void **)&d_Q, sizeof(float) * 5 * (size_t)N));
    CHECK_CUDA(cudaMalloc((void **)&d_b0, sizeof(float) * (size_t)N));
    CHECK_CUDA(cudaMemcpy(d_occ, h_occ, (size_t)N, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d_beacons, h_beacons, sizeof(h_beacons), cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemcpy(d_b0, h_b0, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice));
    CHECK_CUDA(cudaMemset(d_V, 0, sizeof(double) * (size_t)N));

    CHECK_QV(qv_model_build(H, W, P, d_occ, d_beacons, 2, 4, goal, d_cell, NULL));
    memset(&m, 0, sizeof(m));
    m.H = H;
    m.W = W;
    m.pitch = P;
    m.d_cell = d_cell;
    m.num_beacons = 2;
    m.goal = goal;
    m.slip = 0.1f;
    m.accuracy = 0.9f;
    m.discount = 0.95f;
    m.d_cost = NULL;
    m.d_beacons = d_beacons;
    m.sense_range = 4;

    vi_bytes = mdp_value_iterate_workspace_bytes(&m, QV_F64);
    memset(&prm, 0, sizeof(prm));
    prm.depth = 2;
    prm.K = 4;
    prm.seed = seed;
    prm.episode = 0;
    prm.weight_mode = QV_WEIGHT_FREQ;
    prm.leaf_mode = QV_LEAF_FUSED;
    plan_bytes = qv_plan_workspace_bytes(1, &m, &prm);
    if (plan_bytes == 0) {
        fprintf(stderr, "qv_plan_workspace_bytes: %s\n", qv_last_error());
        return 1;
    }
    CHECK_CUDA(cudaMalloc(&d_ws, vi_bytes > plan_bytes ? vi_bytes : plan_bytes));
    CHECK_QV(mdp_value_iterate(&m, QV_F64, 1e-9, 100000, 0, d_V, d_Q, d_ws, vi_bytes, &sweeps, &residual, NULL));
    CHECK_QV(qv_tree_plan(&m, d_Q, d_b0, &prm, d_ws, plan_bytes, &res, NULL));
    /* a refused call returns a status and leaves a message */
    prm.K = 0;
    if (qv_plan_workspace_bytes(1, &m, &prm) != 0) return 2;

    printf("{\"action\": %d, \"value\": %.9g, \"q\": [", res.action, res.value);
    for (i = 0; i < 5; ++i) printf("%s%.9g", i ? ", " : "", res.q[i]);
    printf("], \"nodes\": [%lld, %lld, %lld], \"sweeps\": %d, \"goal\": %d, \"beacons\": [%d, %d]}\n",
           (long long)res.nodes_per_level[0], (long long)res.nodes_per_level[1], (long long)res.nodes_per_level[2],
           sweeps, goal, h_beacons[0], h_beacons[1]);
    cudaFree(d_ws);
    cudaFree(d_b0);
    cudaFree(d_Q);
    cudaFree(d_V);
    cudaFree(d_cell);
    cudaFree(d_beacons);
    cudaFree(d_occ);
    free(h_occ);
    free(h_b0);
    return 0;
}
