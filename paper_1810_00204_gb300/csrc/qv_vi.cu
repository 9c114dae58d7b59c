// qv_vi.cu -- MDP value iteration for the offline QMDP alpha-vectors.
//
// Bellman operator of Eq. 2 on a known state (the MDP baseline of Sec. V-B,
// a contraction as noted for Eq. 7): for a free, non-goal cell x
//   V_{k+1}(x) = max_a sum_y T(x, a, y) [r(y) + gamma V_k(y)],
// which equals max_a [R(x, a) + gamma sum_y T(x, a, y) V_k(y)] because
// R(x, a) = sum_y T(x, a, y) r(y).  Jacobi sweeps; V(goal) = 0.
//
// One persistent cooperative launch runs every sweep.  Each CTA owns a band of
// rows; per sweep it stages the band and its two halo rows of V_k into shared
// memory with one bulk (TMA) copy, writes V_{k+1} for its rows, reduces
// max |V_{k+1} - V_k| with warp shuffles, and meets the other CTAs at a grid
// barrier whose waits are bounded (timeout -> status bit, every CTA exits).
#include <algorithm>

#include "qv_vi_cell.cuh"

namespace qv {


template <typename T>
struct VIArgs {
    int H, W, P;
    const uint16_t *cell;
    const float *cost;
    int goal;
    float slip;
    T gamma;
    T tol;
    int max_sweeps;
    int truncated;
    T *V0;               // caller's buffer (holds V_k for even k)
    T *V1;               // workspace buffer (odd k)
    float *Q;            // [5][H][P]
    T *res_slots;        // [gridDim.x] per-CTA residuals
    VIWork *work;
    int *sweeps_out;     // device: number of sweeps
    T *residual_out;     // device: last residual
    int chunk_rows;      // rows staged per smem chunk
    T *ckpt;             // nullable: V_k stored at every k % every == 0, k < sweeps
    int every;
    unsigned *done;      // [gridDim.x] sweeps completed per CTA
    unsigned *arrive;    // [kResRing] cumulative residual postings per ring slot
    unsigned spin_limit; // polls before a wait on other CTAs gives up
};

// Jacobi sweeps by bands of rows, one band per CTA.  Sweep k reads one halo
// row of each neighbouring band, so it waits only for CTAs i - 1 and i + 1
// to finish sweep k - 1 (progress flags).  The stopping test of sweep j
// needs every CTA's residual; it is taken before sweep j + 2, the first
// sweep that overwrites V_{j+1}, so one sweep may run speculatively past the
// one that converged and is discarded: the result is exactly the first
// V_{k+1} with |V_{k+1} - V_k| < tol.  Truncated runs skip the test.
template <typename T>
__global__ void __launch_bounds__(256) k_value_iteration(VIArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ T s_red[8];
    T *Vs = reinterpret_cast<T *>(smem_raw);  // smem row s holds grid row c0 - 1 + s
    const unsigned nblocks = gridDim.x;
    const int rows_per_cta = (a.H + nblocks - 1) / nblocks;
    const int r_begin = min(a.H, (int)blockIdx.x * rows_per_cta);
    const int r_end = min(a.H, r_begin + rows_per_cta);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const bool trunc = a.truncated > 0;
    const int limit = trunc ? a.truncated : a.max_sweeps;
    int F = -1;    // sweeps in the result, once known
    T res = T(0);  // residual of sweep F - 1
    for (int k = 0; k < limit; ++k) {
        if (!trunc && k >= 2) {
            T r;
            if (!sweep_residual(a, k - 2, r)) return;
            if (r < a.tol) {
                F = k - 1;
                res = r;
                break;
            }
        }
        const T *Vk = (k & 1) ? a.V1 : a.V0;
        T *Vn = (k & 1) ? a.V0 : a.V1;
        if (k > 0 && !wait_neighbours(a.done, k, &a.work->status, a.spin_limit)) return;
        if (a.ckpt && k % a.every == 0) {  // this CTA's rows of V_k
            T *dst = a.ckpt + static_cast<size_t>(k / a.every) * a.H * a.P;
            for (int i = r_begin * a.P + threadIdx.x; i < r_end * a.P; i += blockDim.x) dst[i] = Vk[i];
        }
        T local = T(0);
        for (int c0 = r_begin; c0 < r_end; c0 += a.chunk_rows) {
            const int c1 = min(r_end, c0 + a.chunk_rows);
            if (!stage_rows(a, Vs, Vk, c0, c1, a.P, &bar, phase)) return;
            const int ncell = (c1 - c0) * a.P;
            for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
                const int rr = i / a.P, col = i - rr * a.P;
                const int y = (c0 + rr) * a.P + col;
                const unsigned cw = __ldg(a.cell + y);
                T v = T(0);
                if (QV_CELL_FREE(cw) && y != a.goal) {
                    T q[5];
                    cell_q(a, y, col, cw, Vs + (rr + 1) * a.P, q);
                    v = q[0];
#pragma unroll
                    for (int d = 1; d < 5; ++d) v = q[d] > v ? q[d] : v;
                }
                Vn[y] = v;
                const T diff = fabs(v - Vs[(rr + 1) * a.P + col]);
                local = diff > local ? diff : local;
            }
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!trunc || k == limit - 1) {
            // post this CTA's residual of sweep k
            local = warp_max(local);
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = local;
            __syncthreads();
            if (threadIdx.x == 0) {
                T m = T(0);
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = s_red[w] > m ? s_red[w] : m;
                a.res_slots[static_cast<size_t>(k % kResRing) * nblocks + blockIdx.x] = m;
                __threadfence();
                atomicAdd(a.arrive + k % kResRing, 1u);
            }
        }
        publish_step(a.done, k + 1);
    }
    if (F < 0) {
        // the loop ran to its limit: the last two sweeps' tests are still open
        if (!trunc && limit >= 2) {
            T r;
            if (!sweep_residual(a, limit - 2, r)) return;
            if (r < a.tol) {
                F = limit - 1;
                res = r;
            }
        }
        if (F < 0) {
            T r;
            if (!sweep_residual(a, limit - 1, r)) return;
            F = limit;
            res = r;
        }
    }
    // V_F and its neighbours' halo rows are complete (every CTA finished
    // sweep F - 1); Q = sum_y T (r + gamma V_F)
    if (!wait_neighbours(a.done, F, &a.work->status, a.spin_limit)) return;
    const T *Vf = (F & 1) ? a.V1 : a.V0;
    const size_t plane = static_cast<size_t>(a.H) * a.P;
    for (int c0 = r_begin; c0 < r_end; c0 += a.chunk_rows) {
        const int c1 = min(r_end, c0 + a.chunk_rows);
        if (!stage_rows(a, Vs, Vf, c0, c1, a.P, &bar, phase)) return;
        const int ncell = (c1 - c0) * a.P;
        for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
            const int rr = i / a.P, col = i - rr * a.P;
            const int y = (c0 + rr) * a.P + col;
            const unsigned cw = __ldg(a.cell + y);
            T q[5] = {T(0), T(0), T(0), T(0), T(0)};
            if (QV_CELL_FREE(cw) && y != a.goal) cell_q(a, y, col, cw, Vs + (rr + 1) * a.P, q);
#pragma unroll
            for (int d = 0; d < 5; ++d) a.Q[d * plane + y] = static_cast<float>(q[d]);
            if (F & 1) a.V0[y] = Vs[(rr + 1) * a.P + col];  // the result lives in the caller's buffer
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.sweeps_out = F;
        *a.residual_out = res;
    }
}

template <typename T>
size_t vi_ws_bytes(int H, int P, int nslots) {
    size_t b = sizeof(VIWork);
    b = (b + 255) & ~size_t(255);
    b += static_cast<size_t>(H) * P * sizeof(T);  // second V buffer
    b = (b + 255) & ~size_t(255);
    b += kResRing * nslots * sizeof(T) + sizeof(int) + sizeof(T) + 64;
    b = (b + 255) & ~size_t(255);
    b += nslots * sizeof(unsigned) + 64;  // progress flags, residual arrival counters
    return (b + 255) & ~size_t(255);
}

template <typename T>
qv_status run_vi(const qv_model_t *m, double tol, int max_sweeps, int truncated, T *d_V, float *d_Q,
                 void *d_ws, size_t ws_bytes, int *sweeps_out, double *residual_out, cudaStream_t st,
                 T *d_ckpt = nullptr, int every = 1) {
    const int H = m->H, P = m->pitch;
    // rows staged per chunk: (chunk + 2) rows within a 40 KB budget (at least
    // three rows, with the opt-in for large dynamic shared memory)
    const size_t budget = std::max<size_t>(40 * 1024, 3 * static_cast<size_t>(P) * sizeof(T));
    int chunk = static_cast<int>(budget / (P * sizeof(T))) - 2;
    if (chunk < 1) return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: pitch %d too wide", P);
    size_t smem = static_cast<size_t>(chunk + 2) * P * sizeof(T);
    void *kern = reinterpret_cast<void *>(k_value_iteration<T>);
    if (smem > 40 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    int per_sm = 0;
    if (qv_check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem), "occupancy") !=
        QV_OK)
        return QV_ERR_CUDA;
    if (per_sm < 1) return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: kernel does not fit an SM");
    int grid = std::min(per_sm * qv_num_sms(), 1024);
    grid = std::min(grid, H);  // at least one row per CTA
    const int rows_per_cta = (H + grid - 1) / grid;
    grid = (H + rows_per_cta - 1) / rows_per_cta;
    chunk = std::min(chunk, rows_per_cta);
    smem = static_cast<size_t>(chunk + 2) * P * sizeof(T);
    if (ws_bytes < vi_ws_bytes<T>(H, P, 1024))
        return qv_set_error(QV_ERR_WORKSPACE, "mdp_value_iterate: workspace %zu < %zu bytes", ws_bytes,
                            vi_ws_bytes<T>(H, P, 1024));
    char *ws = static_cast<char *>(d_ws);
    VIWork *work = reinterpret_cast<VIWork *>(ws);
    size_t off = (sizeof(VIWork) + 255) & ~size_t(255);
    T *V1 = reinterpret_cast<T *>(ws + off);
    off = (off + static_cast<size_t>(H) * P * sizeof(T) + 255) & ~size_t(255);
    T *slots = reinterpret_cast<T *>(ws + off);
    int *d_sweeps = reinterpret_cast<int *>(slots + kResRing * 1024);
    T *d_res = reinterpret_cast<T *>(reinterpret_cast<char *>(d_sweeps) + 16);
    const size_t off_flags =
        (off + kResRing * 1024 * sizeof(T) + sizeof(int) + sizeof(T) + 64 + 255) & ~size_t(255);
    unsigned *flags = reinterpret_cast<unsigned *>(ws + off_flags);
    unsigned *arrive = flags + 1024;
    if (qv_check_cuda(cudaMemsetAsync(work, 0, sizeof(VIWork), st), "memset") != QV_OK ||
        qv_check_cuda(cudaMemsetAsync(flags, 0, sizeof(unsigned) * (1024 + 16), st), "memset") != QV_OK)
        return QV_ERR_CUDA;
    VIArgs<T> a;
    a.H = H;
    a.W = m->W;
    a.P = P;
    a.cell = m->d_cell;
    a.cost = m->d_cost;
    a.goal = m->goal;
    a.slip = m->slip;
    a.gamma = static_cast<T>(m->discount);
    a.tol = static_cast<T>(tol);
    a.max_sweeps = max_sweeps;
    a.truncated = truncated;
    a.V0 = d_V;
    a.V1 = V1;
    a.Q = d_Q;
    a.res_slots = slots;
    a.work = work;
    a.sweeps_out = d_sweeps;
    a.residual_out = d_res;
    a.chunk_rows = chunk;
    a.ckpt = d_ckpt;
    a.every = every;
    a.done = flags;
    a.arrive = arrive;
    a.spin_limit = qv_cross_spin_limit();
    void *args[] = {&a};
    if (qv_check_cuda(cudaLaunchCooperativeKernel(kern, grid, 256, args, smem, st), "value iteration launch") !=
        QV_OK)
        return QV_ERR_CUDA;
    VIWork hw;
    int hs = 0;
    T hr = T(0);
    if (qv_check_cuda(cudaMemcpyAsync(&hw, work, sizeof(hw), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&hs, d_sweeps, sizeof(int), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&hr, d_res, sizeof(T), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "value iteration") != QV_OK)
        return QV_ERR_CUDA;
    if (hw.status & kErrTimeout)
        return qv_set_error(QV_ERR_TIMEOUT, "mdp_value_iterate: grid barrier or copy wait timed out");
    if (sweeps_out) *sweeps_out = hs;
    if (residual_out) *residual_out = static_cast<double>(hr);
    if (truncated <= 0 && !(static_cast<double>(hr) < tol))
        return qv_set_error(QV_ERR_NOT_CONVERGED, "mdp_value_iterate: residual %g after %d sweeps",
                            static_cast<double>(hr), hs);
    return QV_OK;
}

}  // namespace qv

extern "C" size_t mdp_value_iterate_workspace_bytes(const qv_model_t *m, int32_t dtype) {
    if (!m) return 0;
    return dtype == QV_F64 ? qv::vi_ws_bytes<double>(m->H, m->pitch, 1024)
                           : qv::vi_ws_bytes<float>(m->H, m->pitch, 1024);
}

extern "C" qv_status mdp_value_iterate(const qv_model_t *m, int32_t dtype, double tol, int32_t max_sweeps,
                                       int32_t truncated, void *d_V, float *d_Q, void *d_ws, size_t ws_bytes,
                                       int32_t *sweeps_out, double *residual_out, qv_stream_t stream) {
    QV_RANGE("mdp_value_iterate");
    if (const qv_status inj = qv_injected_fault("mdp_value_iterate", true)) return inj;
    if (!m || !m->d_cell || !d_V || !d_Q || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: null pointer");
    if (m->H < 1 || m->W < 1 || m->pitch != QV_PITCH(m->W) || m->W > QV_MAX_WIDTH)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: bad grid");
    if (!(m->discount > 0.0f && m->discount < 1.0f) || !(m->slip >= 0.0f && m->slip <= 0.5f))
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: discount or slip out of range");
    if (truncated <= 0 && max_sweeps < 1)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: max_sweeps < 1");
    if ((reinterpret_cast<uintptr_t>(d_V) | reinterpret_cast<uintptr_t>(d_ws)) & 15)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: buffers must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == QV_F64)
        return qv::run_vi<double>(m, tol, max_sweeps, truncated, static_cast<double *>(d_V), d_Q, d_ws, ws_bytes,
                                  sweeps_out, residual_out, st);
    if (dtype == QV_F32)
        return qv::run_vi<float>(m, tol, max_sweeps, truncated, static_cast<float *>(d_V), d_Q, d_ws, ws_bytes,
                                 sweeps_out, residual_out, st);
    return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate: dtype %d", dtype);
}

extern "C" qv_status mdp_value_iterate_checkpointed(const qv_model_t *m, int32_t sweeps, int32_t every, double *d_V,
                                                    float *d_Q, double *d_Vckpt, void *d_ws, size_t ws_bytes,
                                                    qv_stream_t stream) {
    QV_RANGE("mdp_value_iterate_checkpointed");
    if (!m || !m->d_cell || !d_V || !d_Q || !d_Vckpt || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate_checkpointed: null pointer");
    if (m->H < 1 || m->W < 1 || m->pitch != QV_PITCH(m->W) || m->W > QV_MAX_WIDTH)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate_checkpointed: bad grid");
    if (!(m->discount > 0.0f && m->discount < 1.0f) || !(m->slip >= 0.0f && m->slip <= 0.5f))
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate_checkpointed: discount or slip out of range");
    if (sweeps < 1 || every < 1)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate_checkpointed: sweeps %d every %d", sweeps, every);
    if ((reinterpret_cast<uintptr_t>(d_V) | reinterpret_cast<uintptr_t>(d_ws)) & 15)
        return qv_set_error(QV_ERR_INVALID, "mdp_value_iterate_checkpointed: buffers must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // V_0 = 0
    if (qv_check_cuda(cudaMemsetAsync(d_V, 0, sizeof(double) * m->H * m->pitch, st), "memset") != QV_OK)
        return QV_ERR_CUDA;
    return qv::run_vi<double>(m, 0.0, sweeps, sweeps, d_V, d_Q, d_ws, ws_bytes, nullptr, nullptr, st, d_Vckpt,
                              every);
}
