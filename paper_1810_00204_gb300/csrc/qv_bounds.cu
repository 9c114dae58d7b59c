// qv_bounds.cu -- the AEMS bookkeeping of Alg. 5-7 and Eq. 9 over a plan.
//
// Each V-node of the paper carries an upper bound U, a lower bound L, a
// heuristic H (how much its bound gap can move the root) and E, the V-node
// to expand next within its subtree.  The plan computes U; given the lower
// bound of every leaf (V_PBVI of the leaf belief, Alg. 5), these kernels fill
// the other three fields bottom-up, one launch per level, one warp per
// V-node and the five Q-nodes under it:
//   leaf:    L_V = given, H_V = U_V - L_V, E_V = the leaf itself
//   Q-node:  L_Q = R + gamma sum_children w L_V;  the child maximising
//            gamma w H_V (ties: the first in (parent, action, z) order) gives
//            H_Q = gamma w H_V and E_Q = its E_V  (Alg. 6, discounted as U_Q is)
//   V-node:  L_V = max_a L_Q;  with H(b, a) = 1 only for the action that
//            maximises U_Q (Eq. 9, ties to the lowest), H_V = H_Q and
//            E_V = E_Q of that action  (Alg. 7)
// A Q-node's children are found by binary search on (parent, action) in
// the next level, whose nodes are stored in that order.
#include <cstring>

#include "qv_plan_types.cuh"

namespace qv {
namespace {

struct BoundsLevel {
    const int *count;    // device scalar: nodes in the level
    const float *value;  // U_V
    const float *R;      // [n][5]
    const float *UQ;     // [n][5]
    float *LV, *HV;
    int *EV;
    float *LQ, *HQ;      // [n][5]
    int *EQ;             // [n][5]
};

struct BoundsChild {
    const int *count;
    const int *parent, *action;
    const float *weight;
    const float *LV, *HV;
    const int *EV;
};

__global__ void k_bounds_leaf(const int *__restrict__ count, const float *__restrict__ value,
                              const float *__restrict__ leafL, float *__restrict__ LV, float *__restrict__ HV,
                              int *__restrict__ EV) {
    const int n = __ldg(count);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float l = __ldg(leafL + j);
        LV[j] = l;
        HV[j] = __ldg(value + j) - l;
        EV[j] = j;
    }
}

// first index j in [0, n) with key(j) >= k, key(j) = parent(j) * 5 + action(j)
__device__ __forceinline__ int child_lower_bound(const BoundsChild &c, int n, int k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int km = __ldg(c.parent + mid) * 5 + __ldg(c.action + mid);
        if (km < k) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_bounds_level(BoundsLevel v, BoundsChild c, float gamma) {
    const int lane = threadIdx.x & 31;
    const int node = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (node >= __ldg(v.count)) return;
    const int nc = __ldg(c.count);
    float lq[5];
    for (int a = 0; a < 5; ++a) {
        int lo = 0, hi = 0;
        if (lane == 0) {
            lo = child_lower_bound(c, nc, node * 5 + a);
            hi = child_lower_bound(c, nc, node * 5 + a + 1);
        }
        lo = __shfl_sync(0xffffffffu, lo, 0);
        hi = __shfl_sync(0xffffffffu, hi, 0);
        float s = 0.0f, bh = -INFINITY;
        int bj = 0x7fffffff;
        for (int j = lo + lane; j < hi; j += 32) {
            const float w = __ldg(c.weight + j);
            s = fmaf(w, c.LV[j], s);
            const float h = gamma * w * c.HV[j];
            if (h > bh) {  // j ascends within a lane: strict > keeps the first
                bh = h;
                bj = j;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            const float oh = __shfl_xor_sync(0xffffffffu, bh, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (oh > bh || (oh == bh && oj < bj)) {
                bh = oh;
                bj = oj;
            }
        }
        const float r = __ldg(v.R + node * 5 + a);
        lq[a] = hi > lo ? fmaf(gamma, s, r) : r;
        const bool picked = hi > lo && bj < nc;  // (no pick only when every h is NaN)
        if (lane == 0) {
            v.LQ[node * 5 + a] = lq[a];
            v.HQ[node * 5 + a] = picked ? bh : 0.0f;
            v.EQ[node * 5 + a] = picked ? c.EV[bj] : -1;
        }
    }
    __syncwarp();
    if (lane == 0) {
        float lmax = lq[0];
        int au = 0;
        float ubest = __ldg(v.UQ + node * 5);
        for (int a = 1; a < 5; ++a) {
            lmax = fmaxf(lmax, lq[a]);
            const float u = __ldg(v.UQ + node * 5 + a);
            if (u > ubest) {
                ubest = u;
                au = a;
            }
        }
        v.LV[node] = lmax;
        v.HV[node] = v.HQ[node * 5 + au];
        v.EV[node] = v.EQ[node * 5 + au];
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Offsets of level l's arrays in the bounds workspace of episode e.
struct BoundsLayout {
    size_t LV[kMaxD + 1], HV[kMaxD + 1], EV[kMaxD + 1], LQ[kMaxD + 1], HQ[kMaxD + 1], EQ[kMaxD + 1];
    size_t bytes;
};

BoundsLayout bounds_layout(const qv_plan *pl, int e) {
    BoundsLayout L{};
    size_t off = 0;
    const int D = pl->params.depth;
    for (int l = 0; l <= D; ++l) {
        const size_t cap = static_cast<size_t>(pl->eps[e].cap[l]);
        L.LV[l] = off;
        off = a256(off + cap * sizeof(float));
        L.HV[l] = off;
        off = a256(off + cap * sizeof(float));
        L.EV[l] = off;
        off = a256(off + cap * sizeof(int));
        if (l < D) {
            L.LQ[l] = off;
            off = a256(off + 5 * cap * sizeof(float));
            L.HQ[l] = off;
            off = a256(off + 5 * cap * sizeof(float));
            L.EQ[l] = off;
            off = a256(off + 5 * cap * sizeof(int));
        }
    }
    L.bytes = off;
    return L;
}

}  // namespace
}  // namespace qv

extern "C" size_t qv_plan_bounds_workspace_bytes(const qv_plan_t *pl, int32_t e) {
    if (!pl || e < 0 || e >= pl->E) return 0;
    return qv::bounds_layout(pl, e).bytes;
}

extern "C" qv_status qv_plan_bounds_view(const qv_plan_t *pl, int32_t e, int32_t l, void *d_ws,
                                         qv_bounds_view_t *view) {
    if (!pl || !d_ws || !view) return qv_set_error(QV_ERR_INVALID, "qv_plan_bounds_view: null pointer");
    if (e < 0 || e >= pl->E || l < 0 || l > pl->params.depth)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_bounds_view: episode %d level %d out of range", e, l);
    const qv::BoundsLayout L = qv::bounds_layout(pl, e);
    char *ws = static_cast<char *>(d_ws);
    std::memset(view, 0, sizeof(*view));
    view->d_LV = reinterpret_cast<float *>(ws + L.LV[l]);
    view->d_HV = reinterpret_cast<float *>(ws + L.HV[l]);
    view->d_EV = reinterpret_cast<int32_t *>(ws + L.EV[l]);
    if (l < pl->params.depth) {
        view->d_LQ = reinterpret_cast<float *>(ws + L.LQ[l]);
        view->d_HQ = reinterpret_cast<float *>(ws + L.HQ[l]);
        view->d_EQ = reinterpret_cast<int32_t *>(ws + L.EQ[l]);
    }
    return QV_OK;
}

extern "C" qv_status qv_plan_bounds(const qv_plan_t *pl, int32_t e, const float *d_leaf_L, void *d_ws,
                                    size_t ws_bytes, qv_stream_t stream) {
    QV_RANGE("qv_plan_bounds");
    if (!pl || !d_leaf_L || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv_plan_bounds: null pointer");
    if (e < 0 || e >= pl->E) return qv_set_error(QV_ERR_INVALID, "qv_plan_bounds: episode %d out of range", e);
    const qv::BoundsLayout L = qv::bounds_layout(pl, e);
    if (ws_bytes < L.bytes)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_plan_bounds: workspace %zu < %zu bytes", ws_bytes, L.bytes);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_bounds: workspace must be 256-byte aligned");
    const int D = pl->params.depth;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    qv_level_view_t lv[qv::kMaxD + 1];
    for (int l = 0; l <= D; ++l) {
        const qv_status s = qv_plan_level(pl, e, l, &lv[l]);
        if (s != QV_OK) return s;
    }
    qv_bounds_view_t bv[qv::kMaxD + 1];
    for (int l = 0; l <= D; ++l) qv_plan_bounds_view(pl, e, l, d_ws, &bv[l]);
    const float gamma = pl->eps[e].gamma;
    const int capd = lv[D].cap;
    qv::k_bounds_leaf<<<std::max(1, std::min((capd + 255) / 256, 4 * qv_num_sms())), 256, 0, st>>>(
        lv[D].d_count, lv[D].d_value, d_leaf_L, bv[D].d_LV, bv[D].d_HV, bv[D].d_EV);
    for (int l = D - 1; l >= 0; --l) {
        QV_RANGE("qv_plan_bounds", l);
        qv::BoundsLevel v;
        v.count = lv[l].d_count;
        v.value = lv[l].d_value;
        v.R = lv[l].d_R;
        v.UQ = lv[l].d_UQ;
        v.LV = bv[l].d_LV;
        v.HV = bv[l].d_HV;
        v.EV = bv[l].d_EV;
        v.LQ = bv[l].d_LQ;
        v.HQ = bv[l].d_HQ;
        v.EQ = bv[l].d_EQ;
        qv::BoundsChild c;
        c.count = lv[l + 1].d_count;
        c.parent = lv[l + 1].d_parent;
        c.action = lv[l + 1].d_action;
        c.weight = lv[l + 1].d_weight;
        c.LV = bv[l + 1].d_LV;
        c.HV = bv[l + 1].d_HV;
        c.EV = bv[l + 1].d_EV;
        const int cap = lv[l].cap;
        qv::k_bounds_level<<<(cap + 7) / 8, 256, 0, st>>>(v, c, gamma);
    }
    return qv_check_cuda(cudaGetLastError(), "qv_plan_bounds launch");
}
