// qv_bestfirst.cu -- best-first QV-Tree Search, the planning loop of Alg. 1.
//
// Every iteration expands the V-node the root's E points at (Eq. 9, Alg.
// 5-7) and updates it and its ancestors.  The tree lives on the device
// (node arrays, per-Q-node arrays, one belief per V-node); the host only
// issues launches, so an iteration never waits for the host:
//   k_bf_expand    one CTA per action of the chosen node v (read from the
//                  root's E on the device): the predicted belief, R(b, a),
//                  P(z | b, a), K forward samples (the level-synchronous
//                  tree's Philox stream: level = depth of v, path = code of
//                  v * 5 + a), the unique z with their frequencies, and the
//                  children's beliefs tau(b, a, z) in a scratch area
//   leaf_value     U of every scratch child (the upper-bound alpha-vectors)
//   qv_pbvi_value  L of every scratch child (the PBVI vectors)
//   k_bf_update    one warp: the children's ids (creation order: a, then z
//                  ascending), their fields (Alg. 5; a child at the depth
//                  limit is closed, H = 0), the Q-nodes of v (Alg. 6) and v
//                  and every ancestor (Alg. 7 with H(b, a) of Eq. 9)
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
    float *sbelief;           // [5 * cmax][N]
    float *sU, *sL;           // [5 * cmax]
    int *sz, *sf, *sm;        // [5][cmax] z, frequency; [5] unique count
    float *sR;                // [5]
};

// One CTA per action of the node the root's E points at.
__global__ void __launch_bounds__(kBfThreads) k_bf_expand(BfDev d) {
    extern __shared__ float hist[];  // [nz][kBfThreads]
    __shared__ float lut[64];
    __shared__ float s_red[kBfThreads / 32];
    __shared__ float s_P[QV_MAX_BEACONS + 1], s_C[QV_MAX_BEACONS + 1];
    __shared__ int s_cnt[QV_MAX_BEACONS + 1];
    __shared__ int s_go, s_v, s_m;
    const int a = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) {
        const int v = d.E[0];
        const int n = d.state[0];
        const bool stop = d.state[2] != 0 || d.depth[v] >= d.max_depth || n + 5 * d.cmax > d.max_nodes;
        s_go = stop ? 0 : 1;
        s_v = v;
    }
    for (int i = tid; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, d.slip);
    for (int z = 0; z < d.nz; ++z) hist[z * kBfThreads + tid] = 0.0f;
    for (int z = tid; z < d.nz; z += blockDim.x) s_cnt[z] = 0;
    __syncthreads();
    if (!s_go) {
        if (a == 0 && tid == 0) d.state[2] = 1;
        return;
    }
    const int v = s_v;
    const float *b = d.belief + static_cast<size_t>(v) * d.N;
    float *bbar = d.sbelief + static_cast<size_t>(a) * d.cmax * d.N;  // first child slot holds bbar
    float rs = 0.0f;
    for (int y = tid; y < d.N; y += blockDim.x) {
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
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = rs;
    __syncthreads();
    for (int z = tid; z < d.nz; z += blockDim.x) {
        float s = 0.0f;
        for (int t = 0; t < kBfThreads; ++t) s += hist[z * kBfThreads + t];
        s_P[z] = s;
    }
    __syncthreads();
    if (tid == 0) {
        float r = 0.0f;
        for (int w = 0; w < kBfThreads / 32; ++w) r += s_red[w];
        d.sR[a] = r - 100.0f * b[d.goal];  // the goal's own mass stays and earns nothing
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
                ++m;
            }
        d.sm[a] = m;
        s_m = m;
    }
    __syncthreads();
    // children tau(b, a, z) = O(., z) bbar / P(z); the last child first, so
    // the first slot (which holds bbar) is rewritten last
    for (int j = s_m - 1; j >= 0; --j) {
        const int z = d.sz[a * d.cmax + j];
        const float inv = 1.0f / s_P[z];
        float *out = d.sbelief + (static_cast<size_t>(a) * d.cmax + j) * d.N;
        for (int y = tid; y < d.N; y += blockDim.x) {
            const unsigned cw = __ldg(d.cell + y);
            const float w = QV_CELL_FREE(cw) ? (static_cast<int>(QV_CELL_LABEL(cw)) == z ? d.acc : d.eta) : 0.0f;
            out[y] = bbar[y] * w * inv;
        }
        __syncthreads();
    }
}

// Alg. 6 for the five Q-nodes of u and Alg. 7 for u (lane 0 of one warp).
__device__ void bf_update_node(const BfDev &d, int u) {
    for (int a = 0; a < 5; ++a) {
        const int q = u * 5 + a;
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

__global__ void k_bf_update(BfDev d) {
    if (threadIdx.x != 0 || d.state[2]) return;
    const int v = d.E[0];
    int n = d.state[0];
    d.state[3] = n;  // the first child's id, for k_bf_commit
    for (int a = 0; a < 5; ++a) {
        const int q = v * 5 + a;
        d.R[q] = d.sR[a];
        d.first[q] = n;
        d.count[q] = d.sm[a];
        for (int j = 0; j < d.sm[a]; ++j) {
            const int c = n++;
            const int z = d.sz[a * d.cmax + j], s = a * d.cmax + j;
            d.parent[c] = v;
            d.action[c] = a;
            d.obs[c] = z;
            d.depth[c] = d.depth[v] + 1;
            d.weight[c] = static_cast<float>(d.sf[s]) / static_cast<float>(d.K);
            d.code[c] = (d.code[v] * 5ull + static_cast<unsigned long long>(a)) * static_cast<unsigned long long>(d.nz) +
                        static_cast<unsigned long long>(z);
            d.U[c] = d.sU[s];
            d.L[c] = d.sL[s];
            d.Hh[c] = d.depth[c] < d.max_depth ? d.sU[s] - d.sL[s] : 0.0f;
            d.E[c] = c;
            for (int t = c * 5; t < c * 5 + 5; ++t) {  // a leaf's Q-nodes: empty until it is expanded
                d.first[t] = 0;
                d.count[t] = 0;
                d.R[t] = d.UQ[t] = d.LQ[t] = d.HQ[t] = 0.0f;
                d.EQ[t] = -1;
            }
        }
    }
    d.state[0] = n;
    for (int u = v; u >= 0; u = d.parent[u]) bf_update_node(d, u);
    d.expanded[d.state[1]] = v;
    d.state[1] += 1;
}

// One CTA per scratch child: copy its belief to its id.
__global__ void __launch_bounds__(kBfThreads) k_bf_commit(BfDev d, int stopped_before) {
    (void)stopped_before;
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
};

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
    h->bytes = off;
    h->ready = false;
    *out = h;
    return QV_OK;
}

extern "C" size_t qv_bf_workspace_bytes(const qv_bf_t *h) { return h ? h->bytes : 0; }

extern "C" void qv_bf_destroy(qv_bf_t *h) { delete h; }

extern "C" qv_status qv_bf_reset(qv_bf_t *h, const float *d_b0, void *d_ws, size_t ws_bytes, qv_stream_t stream) {
    if (!h || !d_b0 || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv_bf_reset: null pointer");
    if (ws_bytes < h->bytes)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_bf_reset: workspace %zu < %zu bytes", ws_bytes, h->bytes);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_bf_reset: workspace must be 256-byte aligned");
    char *ws = static_cast<char *>(d_ws);
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
    if (!h) return qv_set_error(QV_ERR_INVALID, "qv_bf_run: null pointer");
    if (!h->ready) return qv_set_error(QV_ERR_INVALID, "qv_bf_run: no tree (qv_bf_reset)");
    if (iters < 0) return qv_set_error(QV_ERR_INVALID, "qv_bf_run: iters %d", iters);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    qv::BfDev &d = h->dev;
    const int S = 5 * d.cmax;
    const size_t smem = static_cast<size_t>(d.nz) * qv::kBfThreads * sizeof(float);
    if (smem > 48 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(qv::k_bf_expand, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    for (int t = 0; t < iters; ++t) {
        qv::k_bf_expand<<<5, qv::kBfThreads, smem, st>>>(d);
        qv_status s = leaf_value(&h->model, h->Qu, d.sbelief, S, d.sU, stream);
        if (s == QV_OK) s = qv_pbvi_value(h->pbvi, h->G, h->nG, d.sbelief, S, d.sL, nullptr, stream);
        if (s != QV_OK) return s;
        qv::k_bf_update<<<1, 32, 0, st>>>(d);
        qv::k_bf_commit<<<S, qv::kBfThreads, 0, st>>>(d, 0);
    }
    return qv_check_cuda(cudaGetLastError(), "qv_bf_run launch");
}

extern "C" qv_status qv_bf_read(qv_bf_t *h, qv_bf_result_t *r, qv_stream_t stream) {
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
