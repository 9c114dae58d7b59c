// qv_episode.cu -- closed-loop episodes: the outer loop of Alg. 1 (plan,
// execute the action, receive a measurement, update the belief) for E
// episodes at once on one map.
//
// k_env_step      one thread per episode: the true system's motion outcome
//                 (Sec. II, Eq. 10) and measurement (the sensor model) from
//                 a Philox stream of their own, the step count, success and
//                 the discounted return of Eq. 1
// k_bu_predict    grid (episode, band): the predicted belief of the action
//                 taken and, per band, the total mass and the mass on the
//                 measured label
// k_bu_correct    grid (episode, band): Eq. 3's correction, normalised by
//                 P(z) = eta * total + (accuracy - eta) * mass(z) with the
//                 bands' sums added in band order
// The plan between them is the batched level-synchronous plan; its root
// actions are read on the device, so a whole step needs no host wait.
// k_forward_sample is Alg. 4's ancestral sampler as written (x ~ b,
// x' ~ T, z ~ O, one thread per sample) with the same motion and
// measurement rules.
#include <algorithm>

#include "qv_plan_types.cuh"

namespace qv {
namespace {

constexpr int kEpThreads = 256;
constexpr int kEnvLevel = 254;  // Philox level code of the true system's draws

struct EnvArgs {
    int H, W, P, N, B, goal;
    float slip, acc, eta, gamma;
    const uint16_t *cell;
    const float *cost;
};

EnvArgs env_args(const qv_model_t *m) {
    EnvArgs a;
    a.H = m->H;
    a.W = m->W;
    a.P = m->pitch;
    a.N = m->H * m->pitch;
    a.B = m->num_beacons;
    a.goal = m->goal;
    a.slip = m->slip;
    a.acc = m->accuracy;
    a.eta = (1.0f - m->accuracy) / static_cast<float>(m->num_beacons);
    a.gamma = m->discount;
    a.cell = m->d_cell;
    a.cost = m->d_cost;
    return a;
}

// One motion outcome of action a from cell x (Sec. II, Eq. 10): the
// intended move if u < 1 - 2 eps, the first perpendicular (a + 1) if
// u < 1 - eps, else the second (a + 3), in FP32; a blocked move, staying,
// the goal and occupied cells keep x.
__device__ __forceinline__ int system_move(const EnvArgs &m, int x, int a, float u) {
    const unsigned cw = m.cell[x];
    if (!QV_CELL_FREE(cw) || x == m.goal || a == 4) return x;
    const float fwd = 1.0f - 2.0f * m.slip;
    const int d = u < fwd ? a : (u < fwd + m.slip ? ((a + 1) & 3) : ((a + 3) & 3));
    const int stepd[4] = {-m.P, 1, m.P, -1};
    return ((QV_CELL_BLOCKED(cw) >> d) & 1u) ? x : x + stepd[d];
}

// One measurement at cell y: O(y, .) is the accuracy on y's label and eta
// elsewhere, drawn by the FP32 inverse CDF in ascending z.
__device__ __forceinline__ int system_measure(const EnvArgs &m, int y, float u) {
    const int own = static_cast<int>(QV_CELL_LABEL(m.cell[y]));
    float total = 0.0f;
    for (int z = 0; z <= m.B; ++z) total = total + (z == own ? m.acc : m.eta);
    const float t_u = u * total;
    float run = 0.0f;
    for (int k = 0; k <= m.B; ++k) {
        run = run + (k == own ? m.acc : m.eta);
        if (t_u < run) return k;
    }
    return m.B;
}

__global__ void k_env_step(EnvArgs m, int E, const int *__restrict__ action, int stride, int *__restrict__ state,
                           uint64_t seed, int step, int *__restrict__ obs, int *__restrict__ steps,
                           float *__restrict__ ret, int *__restrict__ done) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    if (done[e]) {
        obs[e] = -1;
        return;
    }
    const int x = state[e];
    const int a = min(max(action[static_cast<size_t>(e) * stride], 0), 4);
    const float um = sample_uniform(seed, static_cast<uint32_t>(e), kEnvLevel, static_cast<uint64_t>(step), 0);
    const float uo = sample_uniform(seed, static_cast<uint32_t>(e), kEnvLevel, static_cast<uint64_t>(step), 1);
    const int y = system_move(m, x, a, um);
    const int z = system_measure(m, y, uo);
    state[e] = y;
    obs[e] = z;
    const float r = (y == m.goal) ? 100.0f : -1.0f - (m.cost ? m.cost[y] : 0.0f);
    ret[e] += powf(m.gamma, static_cast<float>(step)) * r;
    steps[e] += 1;
    if (y == m.goal) done[e] = 1;
}

__global__ void __launch_bounds__(kEpThreads) k_bu_predict(EnvArgs m, const float *__restrict__ Bset,
                                                           const int *__restrict__ action, int stride,
                                                           const int *__restrict__ obs, int band_cells,
                                                           float *__restrict__ bbar, float *__restrict__ part) {
    __shared__ float lut[64];
    __shared__ float s_t[kEpThreads / 32], s_m[kEpThreads / 32];
    const int e = blockIdx.x, band = blockIdx.y, tid = threadIdx.x;
    const int z = obs[e];
    if (z < 0) return;  // the episode has ended
    const int a = min(max(action[static_cast<size_t>(e) * stride], 0), 4);
    for (int i = tid; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, m.slip);
    __syncthreads();
    const float *b = Bset + static_cast<size_t>(e) * m.N;
    float *o = bbar + static_cast<size_t>(e) * m.N;
    const int y0 = band * band_cells, y1 = min(m.N, y0 + band_cells);
    float tot = 0.0f, mz = 0.0f;
    for (int y = y0 + tid; y < y1; y += blockDim.x) {
        const unsigned cw = __ldg(m.cell + y);
        const unsigned in = QV_CELL_INFLOW(cw);
        float nb[4];
        nb[kDirN] = (in & 1u) ? b[y - m.P] : 0.0f;
        nb[kDirE] = (in & 2u) ? b[y + 1] : 0.0f;
        nb[kDirS] = (in & 4u) ? b[y + m.P] : 0.0f;
        nb[kDirW] = (in & 8u) ? b[y - 1] : 0.0f;
        const float p = predict_one(nb, b[y], cw, y == m.goal, m.slip, lut, a);
        o[y] = p;
        if (QV_CELL_FREE(cw)) {
            tot += p;
            if (static_cast<int>(QV_CELL_LABEL(cw)) == z) mz += p;
        }
    }
    for (int k = 16; k > 0; k >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, k);
        mz += __shfl_xor_sync(0xffffffffu, mz, k);
    }
    if ((tid & 31) == 0) {
        s_t[tid >> 5] = tot;
        s_m[tid >> 5] = mz;
    }
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f, mm = 0.0f;
        for (int w = 0; w < kEpThreads / 32; ++w) {
            t += s_t[w];
            mm += s_m[w];
        }
        part[(static_cast<size_t>(e) * gridDim.y + band) * 2] = t;
        part[(static_cast<size_t>(e) * gridDim.y + band) * 2 + 1] = mm;
    }
}

__global__ void __launch_bounds__(kEpThreads) k_bu_correct(EnvArgs m, float *__restrict__ Bset,
                                                           const int *__restrict__ obs, int band_cells,
                                                           const float *__restrict__ bbar,
                                                           const float *__restrict__ part) {
    __shared__ float s_inv;
    const int e = blockIdx.x, band = blockIdx.y, tid = threadIdx.x;
    const int z = obs[e];
    if (z < 0) return;
    if (tid == 0) {
        float t = 0.0f, mm = 0.0f;
        for (int k = 0; k < static_cast<int>(gridDim.y); ++k) {
            t += part[(static_cast<size_t>(e) * gridDim.y + k) * 2];
            mm += part[(static_cast<size_t>(e) * gridDim.y + k) * 2 + 1];
        }
        s_inv = 1.0f / fmaf(m.acc - m.eta, mm, m.eta * t);
    }
    __syncthreads();
    const float inv = s_inv;
    const float *pb = bbar + static_cast<size_t>(e) * m.N;
    float *o = Bset + static_cast<size_t>(e) * m.N;
    const int y0 = band * band_cells, y1 = min(m.N, y0 + band_cells);
    for (int y = y0 + tid; y < y1; y += blockDim.x) {
        const unsigned cw = __ldg(m.cell + y);
        const float w = QV_CELL_FREE(cw) ? (static_cast<int>(QV_CELL_LABEL(cw)) == z ? m.acc : m.eta) : 0.0f;
        o[y] = pb[y] * w * inv;
    }
}

constexpr int kBandCells = 4096;

// Alg. 4 as written, one CTA per (belief, action) and one thread per
// sample: x ~ b by the inverse CDF over the cells in index order (a
// block-wide FP32 prefix sum over tiles of 1024 cells: four consecutive
// cells per thread, warp shuffles, the warps' totals, a carry from tile to
// tile), x' = system_move, z = system_measure.  Sample k uses words 3k,
// 3k + 1, 3k + 2 of the stream of (level, path).
__global__ void __launch_bounds__(kEpThreads) k_forward_sample(EnvArgs m, const float *__restrict__ Bset,
                                                               const int *__restrict__ action,
                                                               const unsigned long long *__restrict__ path,
                                                               int level, uint64_t seed, uint32_t episode, int K,
                                                               float *__restrict__ cdf, int *__restrict__ zout) {
    __shared__ float s_warp[kEpThreads / 32];
    __shared__ float s_carry;
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const float *b = Bset + static_cast<size_t>(j) * m.N;
    float *C = cdf + static_cast<size_t>(j) * m.N;
    if (tid == 0) s_carry = 0.0f;
    __syncthreads();
    // m.N is a multiple of 8 (whole rows of pitch), so every group of four
    // cells is inside the grid and 16-byte aligned
    for (int base = 0; base < m.N; base += 4 * kEpThreads) {
        const int i = base + 4 * tid;
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (i < m.N) {
            const float4 bv = *reinterpret_cast<const float4 *>(b + i);
            const ushort4 cw = *reinterpret_cast<const ushort4 *>(m.cell + i);
            v[0] = QV_CELL_FREE(cw.x) ? bv.x : 0.0f;
            v[1] = QV_CELL_FREE(cw.y) ? bv.y : 0.0f;
            v[2] = QV_CELL_FREE(cw.z) ? bv.z : 0.0f;
            v[3] = QV_CELL_FREE(cw.w) ? bv.w : 0.0f;
        }
        v[1] += v[0];
        v[2] += v[1];
        v[3] += v[2];
        float incl = v[3];  // inclusive scan of the threads' totals within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const float t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        float woff = s_carry;
        for (int w = 0; w < wid; ++w) woff += s_warp[w];
        const float off = woff + incl - v[3];
        if (i < m.N)
            *reinterpret_cast<float4 *>(C + i) = make_float4(off + v[0], off + v[1], off + v[2], off + v[3]);
        __syncthreads();
        if (tid == 0) {
            float t = s_carry;
            for (int w = 0; w < kEpThreads / 32; ++w) t += s_warp[w];
            s_carry = t;
        }
        __syncthreads();
    }
    __syncthreads();
    const float total = C[m.N - 1];
    const int a = min(max(action[j], 0), 4);
    const unsigned long long pth = path[j];
    for (int k = tid; k < K; k += blockDim.x) {
        const float u1 = sample_uniform(seed, episode, level, pth, 3 * k);
        const float u2 = sample_uniform(seed, episode, level, pth, 3 * k + 1);
        const float u3 = sample_uniform(seed, episode, level, pth, 3 * k + 2);
        const float t = u1 * total;
        int lo = 0, hi = m.N - 1;  // first cell with t < C[cell]
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (t < C[mid]) hi = mid;
            else lo = mid + 1;
        }
        const int y = system_move(m, lo, a, u2);
        zout[static_cast<size_t>(j) * K + k] = system_measure(m, y, u3);
    }
}

}  // namespace
}  // namespace qv

extern "C" size_t qv_forward_sample_workspace_bytes(const qv_model_t *m, int32_t n) {
    if (!m || n < 1) return 0;
    return static_cast<size_t>(n) * m->H * m->pitch * sizeof(float);
}

extern "C" qv_status qv_forward_sample(const qv_model_t *m, int32_t n, const float *d_B, const int32_t *d_action,
                                       const uint64_t *d_path, int32_t level, uint64_t seed, uint32_t episode,
                                       int32_t K, int32_t *d_z, void *d_ws, size_t ws_bytes, qv_stream_t stream) {
    QV_RANGE("qv_forward_sample");
    if (!m || !m->d_cell || !d_B || !d_action || !d_path || !d_z || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "qv_forward_sample: null pointer");
    if (n < 0 || K < 0 || level < 0 || level > 255 || m->num_beacons < 1 || m->num_beacons > QV_MAX_BEACONS)
        return qv_set_error(QV_ERR_INVALID, "qv_forward_sample: bad arguments");
    if (n == 0 || K == 0) return QV_OK;
    if (ws_bytes < qv_forward_sample_workspace_bytes(m, n))
        return qv_set_error(QV_ERR_WORKSPACE, "qv_forward_sample: workspace too small");
    if ((reinterpret_cast<uintptr_t>(d_B) | reinterpret_cast<uintptr_t>(d_ws)) & 15 ||
        reinterpret_cast<uintptr_t>(m->d_cell) & 7)
        return qv_set_error(QV_ERR_INVALID, "qv_forward_sample: beliefs and workspace must be 16-byte aligned");
    qv::k_forward_sample<<<n, qv::kEpThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        qv::env_args(m), d_B, d_action, reinterpret_cast<const unsigned long long *>(d_path), level, seed, episode, K,
        static_cast<float *>(d_ws), d_z);
    return qv_check_cuda(cudaGetLastError(), "qv_forward_sample launch");
}

extern "C" const int32_t *qv_plan_actions_device(const qv_plan_t *pl, int32_t *stride) {
    if (!pl) return nullptr;
    if (stride) *stride = static_cast<int32_t>(sizeof(qv::ResultDev) / sizeof(int32_t));
    return reinterpret_cast<const int32_t *>(pl->dev.result);  // the action is the first field
}

extern "C" qv_status qv_env_step(const qv_model_t *m, int32_t E, const int32_t *d_action, int32_t action_stride,
                                 int32_t *d_state, uint64_t seed, int32_t step, int32_t *d_obs, int32_t *d_steps,
                                 float *d_return, int32_t *d_done, qv_stream_t stream) {
    QV_RANGE("qv_env_step");
    if (!m || !m->d_cell || !d_action || !d_state || !d_obs || !d_steps || !d_return || !d_done)
        return qv_set_error(QV_ERR_INVALID, "qv_env_step: null pointer");
    if (E < 0 || action_stride < 1 || step < 0 || m->num_beacons < 1 || m->num_beacons > QV_MAX_BEACONS)
        return qv_set_error(QV_ERR_INVALID, "qv_env_step: bad arguments");
    if (E == 0) return QV_OK;
    qv::k_env_step<<<(E + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(
        qv::env_args(m), E, d_action, action_stride, d_state, seed, step, d_obs, d_steps, d_return, d_done);
    return qv_check_cuda(cudaGetLastError(), "qv_env_step launch");
}

extern "C" size_t qv_belief_update_batched_workspace_bytes(const qv_model_t *m, int32_t E) {
    if (!m || E < 1) return 0;
    const size_t N = static_cast<size_t>(m->H) * m->pitch;
    const size_t nb = (N + qv::kBandCells - 1) / qv::kBandCells;
    return ((E * N * sizeof(float) + 255) & ~size_t(255)) + E * nb * 2 * sizeof(float);
}

extern "C" qv_status qv_belief_update_batched(const qv_model_t *m, int32_t E, float *d_B, const int32_t *d_action,
                                              int32_t action_stride, const int32_t *d_obs, void *d_ws,
                                              size_t ws_bytes, qv_stream_t stream) {
    QV_RANGE("qv_belief_update_batched");
    if (!m || !m->d_cell || !d_B || !d_action || !d_obs || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "qv_belief_update_batched: null pointer");
    if (E < 0 || action_stride < 1) return qv_set_error(QV_ERR_INVALID, "qv_belief_update_batched: bad arguments");
    if (E == 0) return QV_OK;
    if (ws_bytes < qv_belief_update_batched_workspace_bytes(m, E))
        return qv_set_error(QV_ERR_WORKSPACE, "qv_belief_update_batched: workspace too small");
    const size_t N = static_cast<size_t>(m->H) * m->pitch;
    const int nb = static_cast<int>((N + qv::kBandCells - 1) / qv::kBandCells);
    float *bbar = static_cast<float *>(d_ws);
    float *part = reinterpret_cast<float *>(static_cast<char *>(d_ws) + ((E * N * sizeof(float) + 255) & ~size_t(255)));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const qv::EnvArgs a = qv::env_args(m);
    qv::k_bu_predict<<<dim3(E, nb), qv::kEpThreads, 0, st>>>(a, d_B, d_action, action_stride, d_obs, qv::kBandCells,
                                                             bbar, part);
    qv::k_bu_correct<<<dim3(E, nb), qv::kEpThreads, 0, st>>>(a, d_B, d_obs, qv::kBandCells, bbar, part);
    return qv_check_cuda(cudaGetLastError(), "qv_belief_update_batched launch");
}
