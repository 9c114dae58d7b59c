// qv_vi.cu -- MDP value iteration for the offline QMDP alpha-vectors.
//
// Bellman operator of Eq. 2 on a known state (the MDP baseline of Sec. V-B,
// a contraction as noted for Eq. 7): for a free, non-goal cell x
//   V_{k+1}(x) = max_a sum_y T(x, a, y) [r(y) + gamma V_k(y)],
// which equals max_a [R(x, a) + gamma sum_y T(x, a, y) V_k(y)] because
// R(x, a) = sum_y T(x, a, y) r(y).  Jacobi sweeps; V(goal) = 0.
//
// One persistent cooperative launch runs every sweep.  Each CTA owns a band of
// rows.  k_vi_blocked (chosen by a cost model when it is predicted faster)
// stages its band with an s-row halo of V_k into shared memory with one bulk
// (TMA) copy and runs s sweeps there before the next exchange with its
// neighbours; k_value_iteration stages the band and two halo rows every
// sweep.  Both write V_{k+1} for their rows, reduce max |V_{k+1} - V_k| with
// warp shuffles, and wait on other CTAs only with bounded waits (timeout ->
// status bit, every CTA exits).
#include <algorithm>
#include <cstdlib>

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
    // temporally blocked sweeps (k_vi_blocked)
    int s;               // sweeps per exchange (1..kMaxBlock)
    int R;               // rows owned per CTA
    int nh;              // neighbouring CTAs on each side whose rows a block's halo reaches
    T *hist;             // [2 s][H][P] V_k of the last two blocks, plane k mod 2 s
    T *bres;             // [kResRing][kMaxBlock][gridDim.x] per-sweep residuals of a block
};

constexpr int kVIBThreads = 1024;  // threads of a k_vi_blocked CTA

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

// ---------------------------------------------------------------- temporally blocked sweeps
// The same Jacobi iteration with s sweeps per exchange.  CTA i owns rows
// [i R, i R + R); a block of s sweeps stages V_{b s} on rows [i R - s,
// i R + R + s) into shared memory once and runs its s sweeps there, sweep j
// over the owned rows widened by s - 1 - j rows on each side (the reach of
// the sweeps still to come), so the owned rows of V_{b s + s} are exact
// without any exchange inside the block.  Every sweep's owned rows go to the
// plane k mod 2 s of a ring in global memory (the result and checkpoints can
// be any sweep; the block-end plane is what the neighbours stage next) and
// its residual over the owned rows to a per-block slot.  Between blocks a
// CTA waits only for the nh = ceil(s / R) CTAs on each side whose rows its
// halo reads.  The stopping test of block b (the first sweep in it whose
// residual over every CTA is below tol) is taken before block b + 2, the
// first block that reuses b's planes: the result is exactly the first
// V_{k+1} with max |V_{k+1} - V_k| < tol, as in k_value_iteration.

// r(x) for a free cell x (the arrival reward of Sec. V's cost): +100 at the
// goal, -1 - c(x) elsewhere
template <typename T>
__device__ __forceinline__ T arrive_reward(const VIArgs<T> &a, int y) {
    const float c = a.cost ? __ldg(a.cost + y) : 0.0f;
    return (y == a.goal) ? T(100) : T(-1) - T(c);
}

template <typename T>
__global__ void __launch_bounds__(kVIBThreads) k_vi_blocked(VIArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ T s_red[kVIBThreads / 32][kMaxBlock];
    const int s = a.s, R = a.R, P = a.P, H = a.H;
    const int r_begin = static_cast<int>(blockIdx.x) * R, r_end = min(H, r_begin + R);
    const int base = r_begin - s;  // grid row of shared row 0
    const int nrows = R + 2 * s;
    const int glo = max(0, base), ghi = min(H, base + nrows);  // grid rows held
    const size_t nb = static_cast<size_t>(nrows) * P;
    // V_k and the arrival values A_k(y) = r(y) + gamma V_k(y), two of each
    // (ping-pong), the arrival rewards r(y) and the cell words of the rows
    // held (the goal's free bit cleared there: the goal is never updated)
    T *const V0s = reinterpret_cast<T *>(smem_raw), *const V1s = V0s + nb;
    T *const A0s = V0s + 2 * nb, *const A1s = V0s + 3 * nb;
    T *const rws = V0s + 4 * nb;
    uint16_t *cws = reinterpret_cast<uint16_t *>(V0s + 5 * nb);
    const size_t plane = static_cast<size_t>(H) * P;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // division-free cell walk: thread (rsub, c0) visits rows rsub, rsub +
    // rstep, ... and columns c0, c0 + cstep, ...
    const int nt = static_cast<int>(blockDim.x);
    const int rstep = P <= nt ? nt / P : 1;
    const int rsub = P <= nt ? static_cast<int>(threadIdx.x) / P : 0;
    const int c0 = P <= nt ? static_cast<int>(threadIdx.x) - rsub * P : static_cast<int>(threadIdx.x);
    const int cstep = P <= nt ? P : nt;
    const bool active = rsub < rstep;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    // the cell words and arrival rewards of every row held, once (they do not change)
    for (int i = threadIdx.x; i < (ghi - glo) * P; i += blockDim.x) {
        const int y = glo * P + i;
        const uint16_t cw = __ldg(a.cell + y);
        cws[(glo - base) * P + i] = y == a.goal ? static_cast<uint16_t>(cw & 0x7FFFu) : cw;
        rws[(glo - base) * P + i] = arrive_reward(a, y);
    }
    if (a.ckpt)  // V_0
        for (int i = r_begin * P + threadIdx.x; i < r_end * P; i += blockDim.x) a.ckpt[i] = a.V0[i];
    __syncthreads();
    unsigned phase = 0;
    const bool trunc = a.truncated > 0;
    const int limit = trunc ? a.truncated : a.max_sweeps;
    const int nblk = (limit + s - 1) / s;
    int F = -1;    // sweeps in the result, once known
    T res = T(0);  // residual of sweep F - 1
    for (int b = 0; b < nblk; ++b) {
        if (!trunc && b >= 2) {
            int f;
            T r;
            if (!block_test(a, b - 2, s, false, f, r)) return;
            if (f >= 0) {
                F = f + 1;
                res = r;
                break;
            }
        }
        const int k0 = b * s, ns = min(s, limit - k0);
        if (b > 0 && !wait_range(a.done, b, a.nh, &a.work->status, a.spin_limit)) return;
        // stage V_{k0} on the held rows: one bulk copy
        const T *src = b == 0 ? a.V0 : a.hist + static_cast<size_t>(k0 % (2 * s)) * plane;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            fence_proxy_async();
            const unsigned bytes = static_cast<unsigned>((ghi - glo) * P * sizeof(T));
            mbar_arrive_expect_tx(&bar, bytes);
            bulk_copy_g2s(V0s + (glo - base) * P, src + static_cast<size_t>(glo) * P, bytes, &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, phase);
        const int failed = __syncthreads_or(ok ? 0 : 1);
        if (failed) {
            if (threadIdx.x == 0) atomicOr(&a.work->status, kErrTimeout);
            if (!ok) mbar_wait_bounded(&bar, phase);  // let the copy in flight land before leaving
            return;
        }
        phase ^= 1u;
        // A_{k0} on the held rows (read only at free cells)
        if (active)
            for (int row = glo + rsub; row < ghi; row += rstep)
                for (int col = c0; col < P; col += cstep) {
                    const int t = (row - base) * P + col;
                    A0s[t] = rws[t] + a.gamma * V0s[t];
                }
        __syncthreads();
        int cur = 0;
        for (int j = 0; j < ns; ++j) {
            const int k = k0 + j;  // this sweep makes V_{k+1}
            const int ext = ns - 1 - j;
            const int lo = max(0, r_begin - ext), hi = min(H, r_end + ext);
            T *dst = a.hist + static_cast<size_t>((k + 1) % (2 * s)) * plane;
            T *ck = (a.ckpt && (k + 1) % a.every == 0 && k + 1 < limit)
                        ? a.ckpt + static_cast<size_t>((k + 1) / a.every) * plane
                        : nullptr;
            const T *Vc = cur ? V1s : V0s, *Ac = cur ? A1s : A0s;
            T *Vn = cur ? V0s : V1s, *An = cur ? A0s : A1s;
            T lm = T(0);
            if (active)
                for (int row = lo + rsub; row < hi; row += rstep) {
                    const bool own = row >= r_begin && row < r_end;
                    for (int col = c0; col < P; col += cstep) {
                        const int t = (row - base) * P + col;
                        const int y = row * P + col;
                        const unsigned cw = cws[t];
                        T v = T(0);
                        if (QV_CELL_FREE(cw)) {  // free and not the goal
                            T wn[4] = {Ac[t - P], Ac[t + 1], Ac[t + P], Ac[t - 1]};
                            T q[5];
                            q_from_arrivals(QV_CELL_BLOCKED(cw), Ac[t], wn, a.slip, q);
                            v = fmax(fmax(fmax(q[0], q[1]), fmax(q[2], q[3])), q[4]);
                        }
                        Vn[t] = v;
                        An[t] = rws[t] + a.gamma * v;
                        if (own) {
                            const T diff = fabs(v - Vc[t]);
                            lm = diff > lm ? diff : lm;
                            dst[y] = v;
                            if (ck) ck[y] = v;
                        }
                    }
                }
            lm = warp_max(lm);
            if (lane == 0) s_red[wid][j] = lm;
            __syncthreads();
            cur ^= 1;
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        // post the block's residuals (owned rows), then the progress flag
        if (threadIdx.x < ns) {
            T m = T(0);
            for (int w = 0; w < kVIBThreads / 32; ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
            a.bres[(static_cast<size_t>(b % kResRing) * kMaxBlock + threadIdx.x) * gridDim.x + blockIdx.x] = m;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.arrive + b % kResRing, 1u);
        }
        publish_step(a.done, static_cast<unsigned>(b + 1));
    }
    if (F < 0) {
        // the loop ran to its limit: the last two blocks' tests are still open
        for (int bt = max(0, nblk - 2); bt < nblk && F < 0; ++bt) {
            const int ns = min(s, limit - bt * s);
            if (trunc && bt < nblk - 1) continue;
            int f;
            T r;
            if (!block_test(a, bt, ns, trunc, f, r)) return;
            if (f >= 0) {
                F = f + 1;
                res = r;
            } else if (bt == nblk - 1) {
                F = limit;
                res = r;
            }
        }
    }
    // every CTA has posted the block holding V_F, so its owned rows and the
    // neighbours' are in plane F mod 2 s; Q = sum_y T (r + gamma V_F)
    const T *Vf = a.hist + static_cast<size_t>(F % (2 * s)) * plane;
    const int qlo = max(0, r_begin - 1), qhi = min(H, r_end + 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        fence_proxy_async();
        const unsigned bytes = static_cast<unsigned>((qhi - qlo) * P * sizeof(T));
        mbar_arrive_expect_tx(&bar, bytes);
        bulk_copy_g2s(V0s + (qlo - base) * P, Vf + static_cast<size_t>(qlo) * P, bytes, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, phase);
    if (__syncthreads_or(ok ? 0 : 1)) {
        if (threadIdx.x == 0) atomicOr(&a.work->status, kErrTimeout);
        if (!ok) mbar_wait_bounded(&bar, phase);
        return;
    }
    for (int i = threadIdx.x; i < (r_end - r_begin) * P; i += blockDim.x) {
        const int rr = i / P, col = i - rr * P;
        const int row = r_begin + rr;
        const int t = (row - base) * P + col;
        const int y = row * P + col;
        const unsigned cw = cws[t];
        T q[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (QV_CELL_FREE(cw) && y != a.goal) cell_q(a, y, col, cw, V0s + (row - base) * P, q);
#pragma unroll
        for (int d = 0; d < 5; ++d) a.Q[d * plane + y] = static_cast<float>(q[d]);
        a.V0[y] = V0s[t];  // the result lives in the caller's buffer
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
    b = (b + 255) & ~size_t(255);
    b += 2 * kMaxBlock * static_cast<size_t>(H) * P * sizeof(T);  // the blocked sweeps' ring of planes
    b = (b + 255) & ~size_t(255);
    b += static_cast<size_t>(kResRing) * kMaxBlock * nslots * sizeof(T);  // their per-block residuals
    return (b + 255) & ~size_t(255);
}

// Shape of the blocked sweeps: R rows per CTA (one CTA per SM) and s sweeps
// per exchange, from a cost model of one sweep fitted to GB300 timings of
// both kernels on the 20x20, 128x128 and 512x512 maps: the exchange
// (neighbour wait, staging, residual posting) is shared by s sweeps, and a
// sweep computes R + s - 1 rows on average (the halo rows are computed again
// by the neighbours); FP64 issues at 1/64 of the FP32 rate on this part, so
// there the halo costs more.  The one-sweep-per-exchange kernel is modelled
// by its exchange plus its cells per SM, and kept unless the blocked one is
// predicted at least 10 % faster.  The environment variable QVTS_VI_BLOCK
// (1, 2, 4 or 8) forces s; "0" forces the one-sweep-per-exchange kernel.
// False: run k_value_iteration.
template <typename T>
bool vi_block_shape(int H, int P, int nsm, int &G, int &R, int &s, int &nh, size_t &smem) {
    R = (H + nsm - 1) / nsm;
    G = (H + R - 1) / R;
    const char *env = std::getenv("QVTS_VI_BLOCK");
    const int forced = env ? std::atoi(env) : 0;
    if (env && *env && forced == 0) return false;
    const bool f64 = sizeof(T) == 8;
    // ns per sweep: exchange, per cell computed, fixed
    const double xb = f64 ? 6300.0 : 3590.0, cb = f64 ? 4.8 : 0.42, ob = f64 ? 2330.0 : 930.0;
    const double xo = f64 ? 4900.0 : 3900.0, co = f64 ? 13.3 : 0.93;
    const double t_old = xo + co * static_cast<double>(H) * P / nsm;
    double best = 1e30;
    for (int c : {8, 4, 2, 1}) {
        if (forced > 0 && c != forced) continue;
        const int h = (c + R - 1) / R;
        const size_t sm = static_cast<size_t>(R + 2 * c) * P * (5 * sizeof(T) + sizeof(uint16_t));
        if (2 * h > 32 || sm > 200 * 1024) continue;
        const double t = xb / c + cb * static_cast<double>(R + c - 1) * P + ob;
        if (t < best) {
            best = t;
            s = c;
            nh = h;
            smem = sm;
        }
    }
    if (best > 1e29) return false;
    return forced > 0 || best < 0.9 * t_old;
}

template <typename T>
qv_status run_vi(const qv_model_t *m, double tol, int max_sweeps, int truncated, T *d_V, float *d_Q,
                 void *d_ws, size_t ws_bytes, int *sweeps_out, double *residual_out, cudaStream_t st,
                 T *d_ckpt = nullptr, int every = 1) {
    const int H = m->H, P = m->pitch;
    // the blocked sweeps when their shape fits (one co-resident CTA per SM)
    int bG = 0, bR = 0, bs = 0, bnh = 0;
    size_t bsmem = 0;
    bool blocked = vi_block_shape<T>(H, P, qv_num_sms(), bG, bR, bs, bnh, bsmem) && bG <= 1024;
    if (blocked) {
        void *bk = reinterpret_cast<void *>(k_vi_blocked<T>);
        if (qv_check_cuda(cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(bsmem)),
                          "smem attr") != QV_OK)
            return QV_ERR_CUDA;
        int per_sm = 0;
        if (qv_check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bk, kVIBThreads, bsmem),
                          "occupancy") != QV_OK)
            return QV_ERR_CUDA;
        blocked = per_sm >= 1 && bG <= per_sm * qv_num_sms();
    }
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
    const size_t off_hist = (off_flags + 1024 * sizeof(unsigned) + 64 + 255) & ~size_t(255);
    a.hist = reinterpret_cast<T *>(ws + off_hist);
    const size_t off_bres =
        (off_hist + 2 * kMaxBlock * static_cast<size_t>(H) * P * sizeof(T) + 255) & ~size_t(255);
    a.bres = reinterpret_cast<T *>(ws + off_bres);
    a.s = bs;
    a.R = bR;
    a.nh = bnh;
    void *args[] = {&a};
    if (blocked) {
        if (qv_check_cuda(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_vi_blocked<T>), bG, kVIBThreads,
                                                      args, bsmem, st),
                          "value iteration launch") != QV_OK)
            return QV_ERR_CUDA;
    } else if (qv_check_cuda(cudaLaunchCooperativeKernel(kern, grid, 256, args, smem, st),
                             "value iteration launch") != QV_OK) {
        return QV_ERR_CUDA;
    }
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
