// qv_bestfirst.cu -- best-first QV-Tree Search, the planning loop of Alg. 1.
//
// Every iteration expands the V-node the root's E points at (Eq. 9, Alg.
// 5-7) and updates it and its ancestors.  The tree lives on the device
// (node arrays, per-Q-node arrays, one belief per V-node); the host only
// issues launches, so an iteration never waits for the host:
//   k_bf_predict   grid (action, band of cells) on the chosen node v (read
//                  from the root's E on the device): the predicted belief
//                  and each band's mass per label and share of R(b, a)
//   k_bf_sample    one CTA per action: P(z | b, a) from the bands' sums (in
//                  band order), K forward samples (the level-synchronous
//                  tree's Philox stream: level = depth of v, path = code of
//                  v * 5 + a), the unique z with their frequencies, R(b, a)
//   k_bf_children  grid (child slot, band): tau(b, a, z) into a scratch area
//   leaf_value     U of every scratch child (the upper-bound alpha-vectors)
//   qv_pbvi_value  L of every scratch child (the PBVI vectors, reordered
//                  once per search)
//   k_bf_update    one warp: the children's ids (creation order: a, then z
//                  ascending) and fields (Alg. 5; a child at the depth limit
//                  is closed, H = 0), then the Q-nodes (Alg. 6, one lane per
//                  action) and fields (Alg. 7 with H(b, a) of Eq. 9) of v and
//                  every ancestor
//   k_bf_commit    the children's beliefs from the scratch area to their ids
// Planning stops (a device flag; later iterations do nothing) when the node
// to expand lies at the depth limit or the tree could outgrow max_nodes.
#include <algorithm>
#include <cstring>

#include "qv_plan_types.cuh"  // kBoundaryEps

namespace qv {
namespace {

constexpr int kBfThreads = 256;

struct BfDev {
    int H, W, P, N, B, nz, goal, K, cmax, max_depth, max_nodes;
    float slip, acc, eta, gamma;
    uint64_t seed;
    uint32_t episode;
    const uint16_t *cell;
    const float *cost;
    // tree
    int *state;          // [0] nodes, [1] iterations, [2] stopped, [3] node being expanded
    unsigned long long *boundary;
    int *parent, *action, *obs, *depth, *E, *expanded;
    unsigned long long *code;
    float *weight, *U, *L, *Hh;
    float *R, *UQ, *LQ, *HQ;  // [max_nodes][5]
    int *EQ, *first, *count;  // [max_nodes][5]
    float *belief;            // [max_nodes][N]
    // scratch of one expansion
    float *sbelief;           // [5 * cmax][N] children
    float *sbbar;             // [5][N] predicted beliefs
    float *spart;             // [5][nbands][nz + 1] band sums: mass per label, then R's share
    float *sU, *sL, *sP;      // [5 * cmax]: U, L, P(z) of each child
    int *sz, *sf, *sm;        // [5][cmax] z, frequency; [5] unique count
    float *sR;                // [5]
    int band_cells, nbands;
    const int *replay;        // [n_replay] (nullable): node to expand at iteration t when >= 0
    int n_replay;
};

// The V-node iteration t expands: the root's E (Eq. 9), unless the caller
// fixed the choice of this iteration (replay of another implementation's
// choices at near-ties); a fixed id must name an existing node.
__device__ __forceinline__ int bf_target(const BfDev &d) {
    const int t = d.state[1];
    if (d.replay && t < d.n_replay) {
        const int f = __ldg(d.replay + t);
        if (f >= 0 && f < d.state[0]) return f;
    }
    return d.E[0];
}

// The node to expand, or -1 when planning has stopped (every CTA of a
// launch reaches the same answer; CTA 0 records a new stop).
__device__ __forceinline__ int bf_node(const BfDev &d, bool record) {
    const int v = bf_target(d);
    const bool stop = d.state[2] != 0 || d.depth[v] >= d.max_depth || d.state[0] + 5 * d.cmax > d.max_nodes;
    if (stop && record) d.state[2] = 1;
    return stop ? -1 : v;
}

// Grid (action, band): the predicted belief of the band's cells, and the
// band's mass per label and share of sum_y bbar(y) r(y) (one shared-memory
// column per thread, added in a fixed order).
__global__ void __launch_bounds__(kBfThreads) k_bf_predict(BfDev d) {
    extern __shared__ float hist[];  // [nz + 1][kBfThreads]; row nz: reward
    __shared__ float lut[64];
    __shared__ int s_v;
    const int a = blockIdx.x, band = blockIdx.y, tid = threadIdx.x;
    if (tid == 0) s_v = bf_node(d, a == 0 && band == 0);
    for (int i = tid; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, d.slip);
    for (int z = 0; z <= d.nz; ++z) hist[z * kBfThreads + tid] = 0.0f;
    __syncthreads();
    const int v = s_v;
    if (v < 0) return;
    const float *b = d.belief + static_cast<size_t>(v) * d.N;
    float *bbar = d.sbbar + static_cast<size_t>(a) * d.N;
    const int y0 = band * d.band_cells, y1 = min(d.N, y0 + d.band_cells);
    float rs = 0.0f;
    for (int y = y0 + tid; y < y1; y += blockDim.x) {
        const unsigned cw = __ldg(d.cell + y);
        const unsigned in = QV_CELL_INFLOW(cw);
        float nb[4];
        nb[kDirN] = (in & 1u) ? b[y - d.P] : 0.0f;
        nb[kDirE] = (in & 2u) ? b[y + 1] : 0.0f;
        nb[kDirS] = (in & 4u) ? b[y + d.P] : 0.0f;
        nb[kDirW] = (in & 8u) ? b[y - 1] : 0.0f;
        const float p = predict_one(nb, b[y], cw, y == d.goal, d.slip, lut, a);
        bbar[y] = p;
        if (QV_CELL_FREE(cw)) {
            hist[QV_CELL_LABEL(cw) * kBfThreads + tid] += p;
            rs = fmaf(p, stage_reward(true, y == d.goal, d.cost ? __ldg(d.cost + y) : 0.0f), rs);
        }
    }
    hist[d.nz * kBfThreads + tid] = rs;
    __syncthreads();
    float *out = d.spart + (static_cast<size_t>(a) * d.nbands + band) * (d.nz + 1);
    for (int z = tid; z <= d.nz; z += blockDim.x) {
        float s = 0.0f;
        for (int t = 0; t < kBfThreads; ++t) s += hist[z * kBfThreads + t];
        out[z] = s;
    }
}

// One CTA per action: P(z) from the band sums, the K samples, the unique z
// with their frequencies, R(b, a).
__global__ void __launch_bounds__(128) k_bf_sample(BfDev d) {
    __shared__ float s_P[QV_MAX_BEACONS + 2], s_C[QV_MAX_BEACONS + 1];
    __shared__ int s_cnt[QV_MAX_BEACONS + 1];
    __shared__ int s_v;
    const int a = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) s_v = bf_node(d, false);
    for (int z = tid; z < d.nz; z += blockDim.x) s_cnt[z] = 0;
    __syncthreads();
    const int v = s_v;
    if (v < 0) return;
    for (int z = tid; z <= d.nz; z += blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < d.nbands; ++k) s += d.spart[(static_cast<size_t>(a) * d.nbands + k) * (d.nz + 1) + z];
        s_P[z] = s;  // mass of label z; s_P[nz]: sum_y bbar(y) r(y)
    }
    __syncthreads();
    if (tid == 0) {
        d.sR[a] = s_P[d.nz] - 100.0f * d.belief[static_cast<size_t>(v) * d.N + d.goal];  // the goal's own mass earns nothing
        float tot = s_P[d.B];
        for (int z = 0; z < d.B; ++z) tot += s_P[z];
        float run = 0.0f;
        for (int z = 0; z < d.nz; ++z) {
            const float p = fmaf(d.acc - d.eta, s_P[z], d.eta * tot);
            s_P[z] = p;
            run = run + p;
            s_C[z] = run;
        }
    }
    __syncthreads();
    const unsigned long long path = d.code[v] * 5ull + static_cast<unsigned long long>(a);
    for (int k = tid; k < d.K; k += blockDim.x) {
        const float u = sample_uniform(d.seed, d.episode, d.depth[v], path, k);
        const float t_u = u * s_C[d.B];
        int lo = 0, hi = d.B;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (t_u < s_C[mid]) hi = mid;
            else lo = mid + 1;
        }
        const float inv = 1.0f / s_C[d.B];
        const bool near = (lo < d.B && fabsf(u - s_C[lo] * inv) < kBoundaryEps) ||
                          (lo > 0 && fabsf(u - s_C[lo - 1] * inv) < kBoundaryEps);
        if (near) atomicAdd(d.boundary, 1ull);
        atomicAdd(&s_cnt[lo], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int m = 0;
        for (int z = 0; z < d.nz; ++z)
            if (s_cnt[z]) {
                d.sz[a * d.cmax + m] = z;
                d.sf[a * d.cmax + m] = s_cnt[z];
                d.sP[a * d.cmax + m] = s_P[z];
                ++m;
            }
        d.sm[a] = m;
    }
}

// Grid (child slot, band): tau(b, a, z) = O(., z) bbar / P(z) on the band.
__global__ void __launch_bounds__(kBfThreads) k_bf_children(BfDev d) {
    const int s = blockIdx.x, band = blockIdx.y;
    const int a = s / d.cmax, j = s - a * d.cmax;
    if (d.state[2] || j >= d.sm[a]) return;
    const int z = d.sz[s];
    const float inv = 1.0f / d.sP[s];
    const float *bbar = d.sbbar + static_cast<size_t>(a) * d.N;
    float *out = d.sbelief + static_cast<size_t>(s) * d.N;
    const int y0 = band * d.band_cells, y1 = min(d.N, y0 + d.band_cells);
    for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
        const unsigned cw = __ldg(d.cell + y);
        const float w = QV_CELL_FREE(cw) ? (static_cast<int>(QV_CELL_LABEL(cw)) == z ? d.acc : d.eta) : 0.0f;
        out[y] = bbar[y] * w * inv;
    }
}

// Alg. 6 for the five Q-nodes of u (lane a of the warp takes action a) and
// Alg. 7 for u (lane 0).
__device__ void bf_update_node(const BfDev &d, int u, int lane) {
    if (lane < 5) {
        const int q = u * 5 + lane;
        const int c0 = d.first[q], nc = d.count[q];
        float su = 0.0f, sl = 0.0f, bh = 0.0f;
        int be = -1;
        for (int c = c0; c < c0 + nc; ++c) {
            su = fmaf(d.weight[c], d.U[c], su);
            sl = fmaf(d.weight[c], d.L[c], sl);
            const float h = d.gamma * d.weight[c] * d.Hh[c];
            if (be < 0 || h > bh) {
                bh = h;
                be = d.E[c];
            }
        }
        d.UQ[q] = fmaf(d.gamma, su, d.R[q]);
        d.LQ[q] = fmaf(d.gamma, sl, d.R[q]);
        d.HQ[q] = bh;
        d.EQ[q] = be;
    }
    __syncwarp();
    if (lane == 0) {
        int au = 0;
        float lmax = d.LQ[u * 5];
        for (int a = 1; a < 5; ++a) {
            if (d.UQ[u * 5 + a] > d.UQ[u * 5 + au]) au = a;
            lmax = fmaxf(lmax, d.LQ[u * 5 + a]);
        }
        d.U[u] = d.UQ[u * 5 + au];
        d.L[u] = lmax;
        d.Hh[u] = d.HQ[u * 5 + au];
        d.E[u] = d.EQ[u * 5 + au];
    }
    __syncwarp();
}

// One warp: the children's ids and fields, then v and its ancestors.
__global__ void __launch_bounds__(32) k_bf_update(BfDev d) {
    const int lane = threadIdx.x;
    if (d.state[2]) return;
    const int v = bf_target(d);
    const int n = d.state[0];
    int base[6];
    base[0] = 0;
    for (int a = 0; a < 5; ++a) base[a + 1] = base[a] + d.sm[a];
    const int total = base[5];
    for (int t = lane; t < total; t += 32) {
        int a = 0;
        while (t >= base[a + 1]) ++a;
        const int j = t - base[a], s = a * d.cmax + j;
        const int c = n + t, z = d.sz[s];
        d.parent[c] = v;
        d.action[c] = a;
        d.obs[c] = z;
        d.depth[c] = d.depth[v] + 1;
        d.weight[c] = static_cast<float>(d.sf[s]) / static_cast<float>(d.K);
        d.code[c] = (d.code[v] * 5ull + static_cast<unsigned long long>(a)) * static_cast<unsigned long long>(d.nz) +
                    static_cast<unsigned long long>(z);
        d.U[c] = d.sU[s];
        d.L[c] = d.sL[s];
        d.Hh[c] = d.depth[v] + 1 < d.max_depth ? d.sU[s] - d.sL[s] : 0.0f;
        d.E[c] = c;
        for (int q = c * 5; q < c * 5 + 5; ++q) {  // a leaf's Q-nodes: empty until it is expanded
            d.first[q] = 0;
            d.count[q] = 0;
            d.R[q] = d.UQ[q] = d.LQ[q] = d.HQ[q] = 0.0f;
            d.EQ[q] = -1;
        }
    }
    if (lane < 5) {
        d.R[v * 5 + lane] = d.sR[lane];
        d.first[v * 5 + lane] = n + base[lane];
        d.count[v * 5 + lane] = d.sm[lane];
    }
    __syncwarp();
    for (int u = v; u >= 0; u = d.parent[u]) bf_update_node(d, u, lane);
    if (lane == 0) {
        d.state[3] = n;  // the first child's id, for k_bf_commit
        d.state[0] = n + total;
        d.expanded[d.state[1]] = v;
        d.state[1] += 1;
    }
}

// One CTA per scratch child: copy its belief to its id.
__global__ void __launch_bounds__(kBfThreads) k_bf_commit(BfDev d) {
    const int s = blockIdx.x, a = s / d.cmax, j = s - a * d.cmax;
    __shared__ int s_id;
    if (threadIdx.x == 0) {
        int id = -1;
        // the children of this expansion start at state[3]; the update kernel
        // ran only when the expansion did (the stop flag is still clear)
        if (!d.state[2] && j < d.sm[a]) {
            int c = d.state[3];
            for (int t = 0; t < a; ++t) c += d.sm[t];
            id = c + j;
        }
        s_id = id;
    }
    __syncthreads();
    if (s_id < 0) return;
    const float4 *src = reinterpret_cast<const float4 *>(d.sbelief + static_cast<size_t>(s) * d.N);
    float4 *dst = reinterpret_cast<float4 *>(d.belief + static_cast<size_t>(s_id) * d.N);
    for (int i = threadIdx.x; i < (d.N >> 2); i += blockDim.x) dst[i] = src[i];
}

// The root: belief b0 (copied by the host), U and L from the scratch slot 0.
__global__ void k_bf_root(BfDev d) {
    if (threadIdx.x != 0) return;
    d.state[0] = 1;
    d.state[1] = 0;
    d.state[2] = 0;
    d.state[3] = 0;
    *d.boundary = 0ull;
    d.parent[0] = -1;
    d.action[0] = -1;
    d.obs[0] = -1;
    d.depth[0] = 0;
    d.code[0] = 0ull;
    d.weight[0] = 1.0f;
    d.U[0] = d.sU[0];
    d.L[0] = d.sL[0];
    d.Hh[0] = d.max_depth > 0 ? d.sU[0] - d.sL[0] : 0.0f;
    d.E[0] = 0;
    for (int a = 0; a < 5; ++a) {
        d.first[a] = 0;
        d.count[a] = 0;
        d.R[a] = d.UQ[a] = d.LQ[a] = d.HQ[a] = 0.0f;
        d.EQ[a] = -1;
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace qv

struct qv_bf {
    qv_model_t model;
    const float *Qu;
    qv_pbvi_t *pbvi;
    const float *G;
    int nG;
    qv::BfDev dev;
    size_t bytes;
    size_t off[32];
    bool ready;
    void *ws;                           // workspace the device pointers point into
    cudaStream_t gs = nullptr;          // private stream the iteration graph replays on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t graph = nullptr;    // one iteration, captured for the workspace `ws`
};

namespace {

void bf_drop_graph(qv_bf *h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
}

// One iteration's launches.  regather: reorder the PBVI vectors again (the
// first iteration of every qv_bf_run call does, so that calls on the PBVI
// handle in between cannot leave stale vectors or piece tables behind).
qv_status bf_issue(qv_bf *h, cudaStream_t st, bool regather) {
    qv::BfDev &d = h->dev;
    const int S = 5 * d.cmax;
    const size_t smem = static_cast<size_t>(d.nz + 1) * qv::kBfThreads * sizeof(float);
    qv::k_bf_predict<<<dim3(5, d.nbands), qv::kBfThreads, smem, st>>>(d);
    qv::k_bf_sample<<<5, 128, 0, st>>>(d);
    qv::k_bf_children<<<dim3(S, d.nbands), qv::kBfThreads, 0, st>>>(d);
    qv_status s = leaf_value(&h->model, h->Qu, d.sbelief, S, d.sU, st);
    if (s == QV_OK) s = qv_pbvi_value(h->pbvi, regather ? h->G : nullptr, h->nG, d.sbelief, S, d.sL, nullptr, st);
    if (s != QV_OK) return s;
    qv::k_bf_update<<<1, 32, 0, st>>>(d);
    qv::k_bf_commit<<<S, qv::kBfThreads, 0, st>>>(d);
    return qv_check_cuda(cudaGetLastError(), "qv_bf_run launch");
}

}  // namespace

extern "C" qv_status qv_bf_create(const qv_model_t *m, const float *d_Qu, qv_pbvi_t *pbvi, const float *d_G,
                                  int32_t nG, int32_t K, uint64_t seed, uint32_t episode, int32_t max_depth,
                                  int32_t max_nodes, qv_bf_t **out) {
    if (!m || !m->d_cell || !d_Qu || !pbvi || !d_G || !out)
        return qv_set_error(QV_ERR_INVALID, "qv_bf_create: null pointer");
    *out = nullptr;
    if (K < 1 || K > QV_MAX_K || max_depth < 0 || max_depth > 8 || nG < 1 || m->num_beacons < 1 ||
        m->num_beacons > QV_MAX_BEACONS || m->goal < 0 || m->goal >= m->H * m->pitch)
        return qv_set_error(QV_ERR_INVALID, "qv_bf_create: bad arguments (K 1..%d, depth limit 0..8)", QV_MAX_K);
    const int nz = m->num_beacons + 1, cmax = std::min(K, nz);
    // path codes stay below 2^56 (the Philox counter's room): (5 |Z|)^depth
    double room = 1.0;
    for (int l = 0; l < max_depth; ++l) room *= 5.0 * nz;
    if (room >= 7.2e16) return qv_set_error(QV_ERR_INVALID, "qv_bf_create: depth limit %d too deep for %d observations", max_depth, nz);
    if (max_nodes < 1 + 5 * cmax) return qv_set_error(QV_ERR_INVALID, "qv_bf_create: max_nodes %d too small", max_nodes);
    qv_bf *h = new qv_bf();
    h->model = *m;
    h->Qu = d_Qu;
    h->pbvi = pbvi;
    h->G = d_G;
    h->nG = nG;
    qv::BfDev &d = h->dev;
    d.H = m->H;
    d.W = m->W;
    d.P = m->pitch;
    d.N = m->H * m->pitch;
    d.B = m->num_beacons;
    d.nz = nz;
    d.goal = m->goal;
    d.K = K;
    d.cmax = cmax;
    d.max_depth = max_depth;
    d.max_nodes = max_nodes;
    d.slip = m->slip;
    d.acc = m->accuracy;
    d.eta = (1.0f - m->accuracy) / static_cast<float>(m->num_beacons);
    d.gamma = m->discount;
    d.seed = seed;
    d.episode = episode;
    d.cell = m->d_cell;
    d.cost = m->d_cost;
    d.band_cells = 4096;
    d.nbands = (d.N + d.band_cells - 1) / d.band_cells;
    const size_t Mn = max_nodes, N = d.N, S = 5 * cmax;
    size_t off = 0;
    int k = 0;
    auto take = [&](size_t bytes) {
        h->off[k++] = off;
        off = qv::a256(off + bytes);
    };
    take(4 * sizeof(int));                  // 0 state
    take(sizeof(unsigned long long));       // 1 boundary
    take(Mn * sizeof(int));                 // 2 parent
    take(Mn * sizeof(int));                 // 3 action
    take(Mn * sizeof(int));                 // 4 obs
    take(Mn * sizeof(int));                 // 5 depth
    take(Mn * sizeof(int));                 // 6 E
    take(Mn * sizeof(int));                 // 7 expanded
    take(Mn * sizeof(unsigned long long));  // 8 code
    take(Mn * sizeof(float));               // 9 weight
    take(Mn * sizeof(float));               // 10 U
    take(Mn * sizeof(float));               // 11 L
    take(Mn * sizeof(float));               // 12 H
    take(5 * Mn * sizeof(float));           // 13 R
    take(5 * Mn * sizeof(float));           // 14 UQ
    take(5 * Mn * sizeof(float));           // 15 LQ
    take(5 * Mn * sizeof(float));           // 16 HQ
    take(5 * Mn * sizeof(int));             // 17 EQ
    take(5 * Mn * sizeof(int));             // 18 first
    take(5 * Mn * sizeof(int));             // 19 count
    take(Mn * N * sizeof(float));           // 20 belief
    take(S * N * sizeof(float));            // 21 scratch beliefs
    take(S * sizeof(float));                // 22 sU
    take(S * sizeof(float));                // 23 sL
    take(S * sizeof(int));                  // 24 sz
    take(S * sizeof(int));                  // 25 sf
    take(8 * sizeof(int));                  // 26 sm
    take(8 * sizeof(float));                // 27 sR
    take(5 * N * sizeof(float));            // 28 sbbar
    take(5 * static_cast<size_t>(d.nbands) * (nz + 1) * sizeof(float));  // 29 spart
    take(S * sizeof(float));                // 30 sP
    h->bytes = off;
    h->ready = false;
    *out = h;
    return QV_OK;
}

extern "C" size_t qv_bf_workspace_bytes(const qv_bf_t *h) { return h ? h->bytes : 0; }

extern "C" void qv_bf_destroy(qv_bf_t *h) {
    if (!h) return;
    bf_drop_graph(h);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->gs) cudaStreamDestroy(h->gs);
    delete h;
}

extern "C" qv_status qv_bf_reset(qv_bf_t *h, const float *d_b0, void *d_ws, size_t ws_bytes, qv_stream_t stream) {
    QV_RANGE("qv_bf_reset");
    if (!h || !d_b0 || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv_bf_reset: null pointer");
    if (ws_bytes < h->bytes)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_bf_reset: workspace %zu < %zu bytes", ws_bytes, h->bytes);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_bf_reset: workspace must be 256-byte aligned");
    char *ws = static_cast<char *>(d_ws);
    if (h->ws != d_ws) bf_drop_graph(h);  // the graph's pointers were the old workspace's
    h->ws = d_ws;
    qv::BfDev &d = h->dev;
    auto P = [&](int i) { return ws + h->off[i]; };
    d.state = reinterpret_cast<int *>(P(0));
    d.boundary = reinterpret_cast<unsigned long long *>(P(1));
    d.parent = reinterpret_cast<int *>(P(2));
    d.action = reinterpret_cast<int *>(P(3));
    d.obs = reinterpret_cast<int *>(P(4));
    d.depth = reinterpret_cast<int *>(P(5));
    d.E = reinterpret_cast<int *>(P(6));
    d.expanded = reinterpret_cast<int *>(P(7));
    d.code = reinterpret_cast<unsigned long long *>(P(8));
    d.weight = reinterpret_cast<float *>(P(9));
    d.U = reinterpret_cast<float *>(P(10));
    d.L = reinterpret_cast<float *>(P(11));
    d.Hh = reinterpret_cast<float *>(P(12));
    d.R = reinterpret_cast<float *>(P(13));
    d.UQ = reinterpret_cast<float *>(P(14));
    d.LQ = reinterpret_cast<float *>(P(15));
    d.HQ = reinterpret_cast<float *>(P(16));
    d.EQ = reinterpret_cast<int *>(P(17));
    d.first = reinterpret_cast<int *>(P(18));
    d.count = reinterpret_cast<int *>(P(19));
    d.belief = reinterpret_cast<float *>(P(20));
    d.sbelief = reinterpret_cast<float *>(P(21));
    d.sU = reinterpret_cast<float *>(P(22));
    d.sL = reinterpret_cast<float *>(P(23));
    d.sz = reinterpret_cast<int *>(P(24));
    d.sf = reinterpret_cast<int *>(P(25));
    d.sm = reinterpret_cast<int *>(P(26));
    d.sR = reinterpret_cast<float *>(P(27));
    d.sbbar = reinterpret_cast<float *>(P(28));
    d.spart = reinterpret_cast<float *>(P(29));
    d.sP = reinterpret_cast<float *>(P(30));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bN = static_cast<size_t>(d.N) * sizeof(float);
    if (qv_check_cuda(cudaMemsetAsync(d.expanded, 0xff, static_cast<size_t>(d.max_nodes) * sizeof(int), st),
                      "memset") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(d.belief, d_b0, bN, cudaMemcpyDeviceToDevice, st), "copy b0") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(d.sbelief, d_b0, bN, cudaMemcpyDeviceToDevice, st), "copy b0") != QV_OK)
        return QV_ERR_CUDA;
    qv_status s = leaf_value(&h->model, h->Qu, d.sbelief, 1, d.sU, stream);
    if (s == QV_OK) s = qv_pbvi_value(h->pbvi, h->G, h->nG, d.sbelief, 1, d.sL, nullptr, stream);
    if (s != QV_OK) return s;
    qv::k_bf_root<<<1, 32, 0, st>>>(d);
    h->ready = true;
    return qv_check_cuda(cudaGetLastError(), "qv_bf_reset launch");
}

extern "C" qv_status qv_bf_run(qv_bf_t *h, int32_t iters, qv_stream_t stream) {
    QV_RANGE("qv_bf_run");
    if (!h) return qv_set_error(QV_ERR_INVALID, "qv_bf_run: null pointer");
    if (!h->ready) return qv_set_error(QV_ERR_INVALID, "qv_bf_run: no tree (qv_bf_reset)");
    if (iters < 0) return qv_set_error(QV_ERR_INVALID, "qv_bf_run: iters %d", iters);
    if (iters == 0) return QV_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    qv::BfDev &d = h->dev;
    const size_t smem = static_cast<size_t>(d.nz + 1) * qv::kBfThreads * sizeof(float);
    if (smem > 48 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(qv::k_bf_predict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    // the first iteration eagerly on the caller's stream (it also restores the
    // PBVI handle's reordered vectors and piece table the graph reads)
    qv_status s = bf_issue(h, st, true);
    if (s != QV_OK || iters == 1) return s;
    if (!h->gs) {
        if (qv_check_cuda(cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking), "stream") != QV_OK ||
            qv_check_cuda(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming), "event") != QV_OK ||
            qv_check_cuda(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming), "event") != QV_OK)
            return QV_ERR_CUDA;
    }
    if (qv_check_cuda(cudaEventRecord(h->ev_in, st), "event") != QV_OK ||
        qv_check_cuda(cudaStreamWaitEvent(h->gs, h->ev_in, 0), "wait") != QV_OK)
        return QV_ERR_CUDA;
    if (!h->graph) {
        cudaGraph_t g = nullptr;
        if (qv_check_cuda(cudaStreamBeginCapture(h->gs, cudaStreamCaptureModeThreadLocal), "capture") != QV_OK)
            return QV_ERR_CUDA;
        const qv_status cs = bf_issue(h, h->gs, false);
        const cudaError_t ce = cudaStreamEndCapture(h->gs, &g);
        if (cs != QV_OK) {
            if (g) cudaGraphDestroy(g);
            return cs;
        }
        if (qv_check_cuda(ce, "end capture") != QV_OK) return QV_ERR_CUDA;
        const cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (qv_check_cuda(ie, "instantiate") != QV_OK) {
            h->graph = nullptr;
            return QV_ERR_CUDA;
        }
    }
    for (int t = 1; t < iters; ++t)
        if (qv_check_cuda(cudaGraphLaunch(h->graph, h->gs), "graph launch") != QV_OK) return QV_ERR_CUDA;
    if (qv_check_cuda(cudaEventRecord(h->ev_out, h->gs), "event") != QV_OK ||
        qv_check_cuda(cudaStreamWaitEvent(st, h->ev_out, 0), "wait") != QV_OK)
        return QV_ERR_CUDA;
    return QV_OK;
}

extern "C" qv_status qv_bf_set_replay(qv_bf_t *h, const int32_t *d_expand, int32_t n) {
    if (!h) return qv_set_error(QV_ERR_INVALID, "qv_bf_set_replay: null pointer");
    if (n < 0 || (n > 0 && !d_expand)) return qv_set_error(QV_ERR_INVALID, "qv_bf_set_replay: n %d", n);
    h->dev.replay = n > 0 ? d_expand : nullptr;
    h->dev.n_replay = n;
    bf_drop_graph(h);  // the captured iteration holds the old parameters
    return QV_OK;
}

extern "C" qv_status qv_bf_read(qv_bf_t *h, qv_bf_result_t *r, qv_stream_t stream) {
    QV_RANGE("qv_bf_read");
    if (!h || !r) return qv_set_error(QV_ERR_INVALID, "qv_bf_read: null pointer");
    if (!h->ready) return qv_set_error(QV_ERR_INVALID, "qv_bf_read: no tree (qv_bf_reset)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const qv::BfDev &d = h->dev;
    int state[4];
    unsigned long long bd = 0;
    float uq[5], U = 0.f, L = 0.f, Hh = 0.f;
    int E = 0, cnt[5];
    if (qv_check_cuda(cudaMemcpyAsync(state, d.state, sizeof(state), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&bd, d.boundary, sizeof(bd), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(uq, d.UQ, sizeof(uq), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(cnt, d.count, sizeof(cnt), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&U, d.U, sizeof(float), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&L, d.L, sizeof(float), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&Hh, d.Hh, sizeof(float), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&E, d.E, sizeof(int), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "qv_bf_read") != QV_OK)
        return QV_ERR_CUDA;
    std::memset(r, 0, sizeof(*r));
    r->nodes = state[0];
    r->iterations = state[1];
    r->stopped = state[2];
    r->U = U;
    r->L = L;
    r->H = Hh;
    r->E = E;
    r->boundary_samples = static_cast<int64_t>(bd);
    int any = 0;
    for (int a = 0; a < 5; ++a) any += cnt[a];
    r->root_action = -1;
    if (any) {
        r->root_action = 0;
        for (int a = 0; a < 5; ++a) {
            r->q[a] = uq[a];
            if (uq[a] > uq[r->root_action]) r->root_action = a;
        }
    }
    return QV_OK;
}

extern "C" qv_status qv_bf_view(const qv_bf_t *h, qv_bf_view_t *v) {
    if (!h || !v) return qv_set_error(QV_ERR_INVALID, "qv_bf_view: null pointer");
    if (!h->ready) return qv_set_error(QV_ERR_INVALID, "qv_bf_view: no tree (qv_bf_reset)");
    const qv::BfDev &d = h->dev;
    v->max_nodes = d.max_nodes;
    v->d_parent = d.parent;
    v->d_action = d.action;
    v->d_obs = d.obs;
    v->d_depth = d.depth;
    v->d_weight = d.weight;
    v->d_U = d.U;
    v->d_L = d.L;
    v->d_H = d.Hh;
    v->d_E = d.E;
    v->d_R = d.R;
    v->d_UQ = d.UQ;
    v->d_LQ = d.LQ;
    v->d_HQ = d.HQ;
    v->d_EQ = d.EQ;
    v->d_first = d.first;
    v->d_count = d.count;
    v->d_belief = d.belief;
    v->d_expanded = d.expanded;
    return QV_OK;
}
