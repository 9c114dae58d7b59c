// qv_belief.cu -- single-belief primitives: the predict step (numerator of
// Eq. 3 with the blocked-move rule of Eq. 10), the Bayes correction with its
// normaliser P(z | b, a) (Eq. 3), and QMDP leaf values (Eq. 4).
#include <mutex>

#include "qv_common.cuh"

namespace qv {

struct ModelArgs {
    int H, W, P, N, B, goal;
    float slip, acc, eta;
    const uint16_t *cell;
};

__host__ ModelArgs model_args(const qv_model_t *m) {
    ModelArgs a;
    a.H = m->H;
    a.W = m->W;
    a.P = m->pitch;
    a.N = m->H * m->pitch;
    a.B = m->num_beacons;
    a.goal = m->goal;
    a.slip = m->slip;
    a.acc = m->accuracy;
    a.eta = (1.0f - m->accuracy) / static_cast<float>(m->num_beacons);
    a.cell = m->d_cell;
    return a;
}

// One thread per group of 4 cells of a row; neighbours read through L1.
__global__ void __launch_bounds__(256) k_predict(ModelArgs m, const float *__restrict__ b, int action,
                                                 float *__restrict__ out) {
    __shared__ float lut[64];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, m.slip);
    __syncthreads();
    const int P4 = m.P >> 2, ng = m.H * P4;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const int r = g / P4, col = (g - r * P4) << 2, y = r * m.P + col;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 up = r > 0 ? __ldg(reinterpret_cast<const float4 *>(b + y - m.P)) : z4;
        const float4 mid = __ldg(reinterpret_cast<const float4 *>(b + y));
        const float4 dn = r + 1 < m.H ? __ldg(reinterpret_cast<const float4 *>(b + y + m.P)) : z4;
        const float left = col > 0 ? __ldg(b + y - 1) : 0.0f;
        const float right = col + 4 < m.P ? __ldg(b + y + 4) : 0.0f;
        const ushort4 cw4 = __ldg(reinterpret_cast<const ushort4 *>(m.cell + y));
        const float u[4] = {up.x, up.y, up.z, up.w};
        const float mm[6] = {left, mid.x, mid.y, mid.z, mid.w, right};
        const float d[4] = {dn.x, dn.y, dn.z, dn.w};
        const unsigned cws[4] = {cw4.x, cw4.y, cw4.z, cw4.w};
        float res[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const unsigned in = QV_CELL_INFLOW(cws[j]);
            float nb[4], o[5];
            nb[kDirN] = (in & 1u) ? u[j] : 0.0f;
            nb[kDirE] = (in & 2u) ? mm[j + 2] : 0.0f;
            nb[kDirS] = (in & 4u) ? d[j] : 0.0f;
            nb[kDirW] = (in & 8u) ? mm[j] : 0.0f;
            predict_cell(nb, mm[j + 1], cws[j], (y + j) == m.goal, m.slip, lut, o);
            res[j] = o[action];
        }
        *reinterpret_cast<float4 *>(out + y) = make_float4(res[0], res[1], res[2], res[3]);
    }
}

// O(y, z) bbar(y) for the four cells of a float4 group (0 off the free cells).
__device__ __forceinline__ float4 weigh4(const ModelArgs &m, float4 v, ushort4 c, int z) {
    float4 o;
    o.x = QV_CELL_FREE(c.x) ? v.x * (static_cast<int>(QV_CELL_LABEL(c.x)) == z ? m.acc : m.eta) : 0.0f;
    o.y = QV_CELL_FREE(c.y) ? v.y * (static_cast<int>(QV_CELL_LABEL(c.y)) == z ? m.acc : m.eta) : 0.0f;
    o.z = QV_CELL_FREE(c.z) ? v.z * (static_cast<int>(QV_CELL_LABEL(c.z)) == z ? m.acc : m.eta) : 0.0f;
    o.w = QV_CELL_FREE(c.w) ? v.w * (static_cast<int>(QV_CELL_LABEL(c.w)) == z ? m.acc : m.eta) : 0.0f;
    return o;
}

constexpr int kStreamUnroll = 4;  // float4 groups whose loads a thread issues together

// P(z) = sum_y O(y, z) bbar(y): per-CTA partial sums, the last CTA adds them
// in CTA order and writes the scalar.
__global__ void __launch_bounds__(256) k_obs_partial(ModelArgs m, const float *__restrict__ bbar, int z,
                                                     float *__restrict__ partials, unsigned *__restrict__ counter,
                                                     float *__restrict__ pz) {
    __shared__ float s_red[8];
    __shared__ int s_last;
    const float4 *b4 = reinterpret_cast<const float4 *>(bbar);
    const ushort4 *c4 = reinterpret_cast<const ushort4 *>(m.cell);
    const int ng = m.N >> 2, stride = gridDim.x * blockDim.x;
    float acc = 0.0f;
    for (int g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < ng; g0 += kStreamUnroll * stride) {
        float4 v[kStreamUnroll];
        ushort4 c[kStreamUnroll];
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) {
            const int g = g0 + u * stride;
            v[u] = g < ng ? __ldcs(b4 + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            c[u] = g < ng ? __ldg(c4 + g) : make_ushort4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) {
            const float4 o = weigh4(m, v[u], c[u], z);
            acc += (o.x + o.y) + (o.z + o.w);
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
        partials[blockIdx.x] = t;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        float t = 0.0f;
        for (unsigned i = 0; i < gridDim.x; ++i) t += __ldcg(partials + i);
        *pz = t;
        *counter = 0u;
    }
}

__global__ void __launch_bounds__(256) k_correct_scale(ModelArgs m, const float *__restrict__ bbar, int z,
                                                       const float *__restrict__ pz, float *__restrict__ out) {
    const float inv = 1.0f / __ldcg(pz);
    const float4 *b4 = reinterpret_cast<const float4 *>(bbar);
    const ushort4 *c4 = reinterpret_cast<const ushort4 *>(m.cell);
    float4 *o4 = reinterpret_cast<float4 *>(out);
    const int ng = m.N >> 2, stride = gridDim.x * blockDim.x;
    for (int g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < ng; g0 += kStreamUnroll * stride) {
        float4 v[kStreamUnroll];
        ushort4 c[kStreamUnroll];
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) {
            const int g = g0 + u * stride;
            v[u] = g < ng ? __ldcs(b4 + g) : make_float4(0.f, 0.f, 0.f, 0.f);
            c[u] = g < ng ? __ldg(c4 + g) : make_ushort4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) {
            const int g = g0 + u * stride;
            if (g < ng) {
                const float4 o = weigh4(m, v[u], c[u], z);
                __stcs(o4 + g, make_float4(o.x * inv, o.y * inv, o.z * inv, o.w * inv));
            }
        }
    }
}

// One CTA of kLeafThreads per belief: max_a sum_y b(y) Q[a][y], with the
// loads of kStreamUnroll float4 columns issued before their arithmetic.
constexpr int kLeafThreads = 1024;
__global__ void __launch_bounds__(kLeafThreads) k_leaf_prim(ModelArgs m, const float *__restrict__ Q,
                                                            const float *__restrict__ b, float *__restrict__ value) {
    __shared__ float s_red[kLeafThreads / 32][5];
    const float4 *bi = reinterpret_cast<const float4 *>(b + static_cast<long long>(blockIdx.x) * m.N);
    const float4 *q4 = reinterpret_cast<const float4 *>(Q);
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const int n4 = m.N >> 2;
    for (int i0 = threadIdx.x; i0 < n4; i0 += kStreamUnroll * blockDim.x) {
        float4 v[kStreamUnroll];
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) {
            const int i = i0 + u * blockDim.x;
            v[u] = i < n4 ? __ldcs(bi + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kStreamUnroll; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= n4) break;
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                const float4 q = __ldg(q4 + static_cast<long long>(a) * n4 + i);
                acc[a] = fmaf(v[u].x, q.x, fmaf(v[u].y, q.y, fmaf(v[u].z, q.z, fmaf(v[u].w, q.w, acc[a]))));
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        const float t = warp_sum(acc[a]);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5][a] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float best = -3.402823466e38f;
        for (int a = 0; a < 5; ++a) {
            float t = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w][a];
            best = t > best ? t : best;
        }
        value[blockIdx.x] = best;
    }
}

constexpr int kCorrectBlocks = 512;

qv_status check_model(const qv_model_t *m, const char *who) {
    if (!m || !m->d_cell) return qv_set_error(QV_ERR_INVALID, "%s: null model", who);
    if (m->H < 1 || m->W < 1 || m->W > QV_MAX_WIDTH || m->pitch != QV_PITCH(m->W))
        return qv_set_error(QV_ERR_INVALID, "%s: bad grid %dx%d pitch %d", who, m->H, m->W, m->pitch);
    if (m->num_beacons < 1 || m->num_beacons > QV_MAX_BEACONS)
        return qv_set_error(QV_ERR_INVALID, "%s: B=%d", who, m->num_beacons);
    if (!(m->slip >= 0.f && m->slip <= 0.5f) || !(m->accuracy > 0.f && m->accuracy <= 1.f))
        return qv_set_error(QV_ERR_INVALID, "%s: slip/accuracy out of range", who);
    return QV_OK;
}

}  // namespace qv

extern "C" qv_status belief_predict(const qv_model_t *m, const float *d_b, int32_t action, float *d_bbar,
                                    qv_stream_t stream) {
    QV_RANGE("belief_predict");
    qv_status st = qv_injected_fault("belief_predict", false);
    if (st != QV_OK) return st;
    st = qv::check_model(m, "belief_predict");
    if (st != QV_OK) return st;
    if (!d_b || !d_bbar) return qv_set_error(QV_ERR_INVALID, "belief_predict: null pointer");
    if (action < 0 || action >= QV_NUM_ACTIONS) return qv_set_error(QV_ERR_INVALID, "belief_predict: action %d", action);
    if ((reinterpret_cast<uintptr_t>(d_b) | reinterpret_cast<uintptr_t>(d_bbar)) & 15)
        return qv_set_error(QV_ERR_INVALID, "belief_predict: buffers must be 16-byte aligned");
    const qv::ModelArgs a = qv::model_args(m);
    const int ng = a.H * (a.P / 4);
    const int grid = std::max(1, std::min((ng + 255) / 256, 8 * qv_num_sms()));
    qv::k_predict<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, d_b, action, d_bbar);
    return qv_check_cuda(cudaGetLastError(), "belief_predict launch");
}

extern "C" size_t belief_correct_workspace_bytes(const qv_model_t *) {
    return sizeof(float) * qv::kCorrectBlocks + 256;
}

extern "C" qv_status belief_correct(const qv_model_t *m, const float *d_bbar, int32_t z, float *d_bout, float *d_pz,
                                    void *d_ws, size_t ws_bytes, qv_stream_t stream) {
    QV_RANGE("belief_correct");
    if (const qv_status inj = qv_injected_fault("belief_correct", true)) return inj;
    qv_status st = qv::check_model(m, "belief_correct");
    if (st != QV_OK) return st;
    if (!d_bbar || !d_bout || !d_pz || !d_ws) return qv_set_error(QV_ERR_INVALID, "belief_correct: null pointer");
    if (z < 0 || z > m->num_beacons) return qv_set_error(QV_ERR_INVALID, "belief_correct: z %d", z);
    if (((reinterpret_cast<uintptr_t>(d_bbar) | reinterpret_cast<uintptr_t>(d_bout)) & 15) ||
        (reinterpret_cast<uintptr_t>(m->d_cell) & 7))
        return qv_set_error(QV_ERR_INVALID, "belief_correct: beliefs must be 16-byte aligned, cell words 8-byte");
    if (ws_bytes < belief_correct_workspace_bytes(m))
        return qv_set_error(QV_ERR_WORKSPACE, "belief_correct: workspace %zu bytes too small", ws_bytes);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const qv::ModelArgs a = qv::model_args(m);
    float *partials = static_cast<float *>(d_ws);
    unsigned *counter = reinterpret_cast<unsigned *>(static_cast<char *>(d_ws) + sizeof(float) * qv::kCorrectBlocks);
    const int grid = std::max(1, std::min((a.N + 255) / 256, qv::kCorrectBlocks));
    if (qv_check_cuda(cudaMemsetAsync(counter, 0, sizeof(unsigned), cs), "belief_correct memset") != QV_OK)
        return QV_ERR_CUDA;
    qv::k_obs_partial<<<grid, 256, 0, cs>>>(a, d_bbar, z, partials, counter, d_pz);
    qv::k_correct_scale<<<grid, 256, 0, cs>>>(a, d_bbar, z, d_pz, d_bout);
    return qv_check_cuda(cudaGetLastError(), "belief_correct launch");
}

// ---------------------------------------------------------------- no-allocation variant
// belief_correct_noalloc runs the two kernels above with their scratch (the
// per-block partial sums and the arrival counter) in a file-scope device
// array instead of a caller workspace.  One block per kNoAllocCellsPerBlock
// cells, so the array's kNoAllocBlocks partial sums bound the grid size.
namespace qv {
constexpr int kNoAllocBlocks = 4096;
constexpr int kNoAllocCellsPerBlock = 1024;
static_assert(static_cast<long long>(kNoAllocBlocks) * kNoAllocCellsPerBlock == QV_NOALLOC_MAX_CELLS,
              "QV_NOALLOC_MAX_CELLS follows the scratch capacity");
// [0, kNoAllocBlocks): partial sums; [kNoAllocBlocks]: the arrival counter.
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocBlocks + 64];
}  // namespace qv

namespace {
std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
float *g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device pointer).
qv_status noalloc_scratch(float **out) {
    int dev = 0;
    if (qv_check_cuda(cudaGetDevice(&dev), "belief_correct_noalloc: cudaGetDevice") != QV_OK) return QV_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return qv_set_error(QV_ERR_INVALID, "belief_correct_noalloc: device ordinal %d unsupported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (qv_check_cuda(cudaGetSymbolAddress(&p, qv::g_noalloc_scratch),
                          "belief_correct_noalloc: cudaGetSymbolAddress") != QV_OK)
            return QV_ERR_CUDA;
        g_noalloc_addr[dev] = static_cast<float *>(p);
    }
    *out = g_noalloc_addr[dev];
    return QV_OK;
}

// After a failed call the cached address may belong to a context that no
// longer exists: drop it, so that the next call on the device looks it up
// again.
void noalloc_forget() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    g_noalloc_addr[dev] = nullptr;
}
}  // namespace

extern "C" qv_status belief_correct_noalloc(const qv_model_t *m, const float *d_bbar, int32_t z, float *d_bout,
                                            float *d_pz, qv_stream_t stream) {
    qv_status st = qv::check_model(m, "belief_correct_noalloc");
    if (st != QV_OK) return st;
    if (!d_bbar || !d_bout || !d_pz) return qv_set_error(QV_ERR_INVALID, "belief_correct_noalloc: null pointer");
    if (z < 0 || z > m->num_beacons) return qv_set_error(QV_ERR_INVALID, "belief_correct_noalloc: z %d", z);
    if (((reinterpret_cast<uintptr_t>(d_bbar) | reinterpret_cast<uintptr_t>(d_bout)) & 15) ||
        (reinterpret_cast<uintptr_t>(m->d_cell) & 7))
        return qv_set_error(QV_ERR_INVALID,
                            "belief_correct_noalloc: beliefs must be 16-byte aligned, cell words 8-byte");
    const long long cells = static_cast<long long>(m->H) * m->pitch;
    if (cells > QV_NOALLOC_MAX_CELLS)
        return qv_set_error(QV_ERR_INVALID,
                            "belief_correct_noalloc: %lld cells exceed the static scratch limit of %d cells",
                            cells, QV_NOALLOC_MAX_CELLS);
    float *scratch = nullptr;
    st = noalloc_scratch(&scratch);
    if (st != QV_OK) return st;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + qv::kNoAllocBlocks);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const qv::ModelArgs a = qv::model_args(m);
    const int grid = static_cast<int>(std::max<long long>(
        1, (cells + qv::kNoAllocCellsPerBlock - 1) / qv::kNoAllocCellsPerBlock));
    // the arrival counter must start at zero; the partial sums are overwritten
    if (qv_check_cuda(cudaMemsetAsync(counter, 0, sizeof(unsigned), cs), "belief_correct_noalloc memset") != QV_OK) {
        noalloc_forget();
        return QV_ERR_CUDA;
    }
    qv::k_obs_partial<<<grid, 256, 0, cs>>>(a, d_bbar, z, scratch, counter, d_pz);
    qv::k_correct_scale<<<grid, 256, 0, cs>>>(a, d_bbar, z, d_pz, d_bout);
    st = qv_check_cuda(cudaGetLastError(), "belief_correct_noalloc launch");
    if (st != QV_OK) noalloc_forget();
    return st;
}

extern "C" qv_status leaf_value(const qv_model_t *m, const float *d_Q, const float *d_b, int32_t n, float *d_value,
                                qv_stream_t stream) {
    QV_RANGE("leaf_value");
    qv_status st = qv::check_model(m, "leaf_value");
    if (st != QV_OK) return st;
    if (!d_Q || !d_b || !d_value) return qv_set_error(QV_ERR_INVALID, "leaf_value: null pointer");
    if (n < 0) return qv_set_error(QV_ERR_INVALID, "leaf_value: n %d", n);
    if (n == 0) return QV_OK;
    if ((reinterpret_cast<uintptr_t>(d_Q) | reinterpret_cast<uintptr_t>(d_b)) & 15)
        return qv_set_error(QV_ERR_INVALID, "leaf_value: buffers must be 16-byte aligned");
    qv::k_leaf_prim<<<n, qv::kLeafThreads, 0, static_cast<cudaStream_t>(stream)>>>(qv::model_args(m), d_Q, d_b,
                                                                                     d_value);
    return qv_check_cuda(cudaGetLastError(), "leaf_value launch");
}
