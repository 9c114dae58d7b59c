// qv_fib.cu -- the Fast Informed Bound alpha-vectors (Sec. IV-A, Eq. 7).
//
// FIB keeps one alpha-vector per action and iterates Eq. 7,
//   alpha'^a(x) = R(x, a) + gamma sum_z max_a' sum_x' O(x', z) T(x, a, x') alpha^a'(x'),
// a monotone contraction, by Jacobi sweeps from alpha_0 = 0.  On the grid
// T(x, a, .) reaches at most three cells (the intended move and the two
// perpendicular slips, blocked moves staying put, Eq. 10), and O(x', z) is
// the sensor accuracy on the label of x' and eta = (1 - accuracy) / B on
// every other observation.  So for one (x, a) only the (at most three)
// labels of the reachable cells differ from eta: with S_a' = sum_x' T
// alpha^a'(x') and G_{l,a'} the part of that sum over the reached cells
// labelled l,
//   sum_z max_a' (...) = sum_{l reached} max_a' [eta S_a' + (acc - eta) G_{l,a'}]
//                      + (|Z| - #labels reached) eta max_a' S_a'.
// That turns the O(|A|^2 |X|^2 |Z|) sweep of the paper's statement into
// O(|X| |A|^2) work, 25 values read per cell: the sweep is a memory-bound
// stencil like the value iteration's, and runs on the same machinery -- one
// persistent cooperative launch, one band of rows per CTA, each band and its
// halo rows staged with one bulk (TMA) copy, neighbour progress flags, and
// the stopping test lagged by one sweep.  Within a sweep the five planes of
// a row are contiguous ([H][5][pitch]) so that one bulk copy stages all of
// them.
#include <algorithm>
#include <cstdlib>

#include "qv_vi_cell.cuh"

namespace qv {

template <typename T>
struct FibArgs {
    int H, W, P;
    const uint16_t *cell;
    const float *cost;
    int goal;
    float slip;
    T gamma;
    T tol;
    T acc;               // alpha
    T eta;               // (1 - alpha) / B
    int nz;              // |Z| = B + 1
    int max_sweeps;
    int truncated;
    T *A0;               // [H][5][P] alpha_k for even k
    T *A1;               // [H][5][P] alpha_k for odd k
    T *alpha_out;        // nullable [5][H][P]
    float *Q;            // [5][H][P]
    T *res_slots;        // [kResRing][gridDim.x] per-CTA residuals
    VIWork *work;
    int *sweeps_out;
    T *residual_out;
    int chunk_rows;
    unsigned *done;      // [gridDim.x] sweeps completed per CTA
    unsigned *arrive;    // [kResRing] cumulative residual postings per ring slot
    unsigned spin_limit;
    // temporally blocked sweeps (k_fib_blocked)
    int s;               // sweeps per exchange (1..kMaxBlock)
    int R;               // rows owned per CTA
    int nh;              // neighbouring CTAs on each side whose rows a block's halo reaches
    T *hist;             // [2 s][H][5][P] alpha_k of the last two blocks, plane k mod 2 s
    T *bres;             // [kResRing][kMaxBlock][gridDim.x] per-sweep residuals of a block
};

constexpr int kFIBThreads = 512;  // threads of a k_fib_blocked CTA

template <typename T>
__device__ __forceinline__ T fib_stage_reward(const FibArgs<T> &a, int y) {
    const float c = a.cost ? __ldg(a.cost + y) : 0.0f;
    return (y == a.goal) ? T(100) : T(-1) - T(c);
}

template <typename T>
__device__ __forceinline__ T fib_core(const FibArgs<T> &a, const T (&al)[5][5], const unsigned (&lab)[5],
                                      const T (&r)[5], T out[5]);

// Eq. 7 for the five actions of a free, non-goal cell y; `rowp` points at
// y's staged row (five planes of P values each, rows 5P apart).  Returns
// max_a |alpha'^a(y) - alpha^a(y)|.
template <typename T>
__device__ __forceinline__ T fib_cell(const FibArgs<T> &a, int y, int col, unsigned cw, const T *rowp,
                                      T out[5]) {
    const int P = a.P;
    const unsigned blk = QV_CELL_BLOCKED(cw);
    // the cells reachable from y: index 0..3 = the move N E S W (y itself when
    // blocked, Eq. 10), 4 = y
    T al[5][5];
    unsigned lab[5];
    T r[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) al[4][b] = rowp[b * P + col];
    lab[4] = QV_CELL_LABEL(cw);
    r[4] = fib_stage_reward(a, y);
    const int drow[4] = {-5 * P, 0, 5 * P, 0};
    const int dcol[4] = {0, 1, 0, -1};
    const int dy[4] = {-P, 1, P, -1};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        if (blk & (1u << d)) {
#pragma unroll
            for (int b = 0; b < 5; ++b) al[d][b] = al[4][b];
            lab[d] = lab[4];
            r[d] = r[4];
        } else {
            const T *q = rowp + drow[d] + col + dcol[d];
#pragma unroll
            for (int b = 0; b < 5; ++b) al[d][b] = q[b * P];
            lab[d] = QV_CELL_LABEL(__ldg(a.cell + y + dy[d]));
            r[d] = fib_stage_reward(a, y + dy[d]);
        }
    }
    return fib_core(a, al, lab, r, out);
}

// Eq. 7's backup of one free, non-goal cell from the alpha values al[d][b]
// at the cell move d reaches (d = 4: the cell itself; a blocked move
// reaches the cell itself, Eq. 10), their labels and their arrival rewards;
// returns max_a |alpha'^a - alpha^a| at the cell.
template <typename T>
__device__ __forceinline__ T fib_core(const FibArgs<T> &a, const T (&al)[5][5], const unsigned (&lab)[5],
                                      const T (&r)[5], T out[5]) {
    const T fwd = T(1) - T(2) * T(a.slip), eps = T(a.slip);
    const T dlt = a.acc - a.eta;
    T diff = T(0);
#pragma unroll
    for (int act = 0; act < 5; ++act) {
        // successors i0 (intended), i1, i2 (perpendicular slips) with their
        // probabilities; staying reaches y alone
        const int i0 = act < 4 ? act : 4;
        const int i1 = act < 4 ? ((act + 1) & 3) : 4;
        const int i2 = act < 4 ? ((act + 3) & 3) : 4;
        const T p0 = act < 4 ? fwd : T(1);
        const T p1 = act < 4 ? eps : T(0);
        const T p2 = act < 4 ? eps : T(0);
        // distinct labels among the three: group 0 is i0's label, group 1
        // i1's when it differs, group 2 i2's when it differs from both
        const bool e10 = lab[i1] == lab[i0];
        const bool e20 = lab[i2] == lab[i0];
        const bool e21 = lab[i2] == lab[i1];
        const bool n1 = !e10;
        const bool n2 = !e20 && !e21;
        T best = -INFINITY, t0 = -INFINITY, t1 = -INFINITY, t2 = -INFINITY;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const T u0 = p0 * al[i0][b], u1 = p1 * al[i1][b], u2 = p2 * al[i2][b];
            const T S = u0 + u1 + u2;
            const T g0 = u0 + (e10 ? u1 : T(0)) + (e20 ? u2 : T(0));
            const T g1 = u1 + (e21 ? u2 : T(0));
            const T base = a.eta * S;
            best = S > best ? S : best;
            const T v0 = base + dlt * g0, v1 = base + dlt * g1, v2 = base + dlt * u2;
            t0 = v0 > t0 ? v0 : t0;
            t1 = v1 > t1 ? v1 : t1;
            t2 = v2 > t2 ? v2 : t2;
        }
        const int m = 1 + (n1 ? 1 : 0) + (n2 ? 1 : 0);
        const T sz = t0 + (n1 ? t1 : T(0)) + (n2 ? t2 : T(0)) + T(a.nz - m) * a.eta * best;
        const T R = p0 * r[i0] + p1 * r[i1] + p2 * r[i2];
        out[act] = R + a.gamma * sz;
        const T dd = fabs(out[act] - al[4][act]);
        diff = dd > diff ? dd : diff;
    }
    return diff;
}

// Jacobi sweeps of Eq. 7 by bands of rows, one band per CTA; the same
// schedule as the value iteration (k_value_iteration): sweep k waits for the
// neighbouring bands to finish sweep k - 1, and the test of sweep j runs
// before sweep j + 2, so the result is the first alpha_{k+1} with
// max |alpha_{k+1} - alpha_k| < tol (or alpha_truncated).
template <typename T>
__global__ void __launch_bounds__(256) k_fib_iteration(FibArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ T s_red[8];
    T *As = reinterpret_cast<T *>(smem_raw);  // smem row s holds grid row c0 - 1 + s, [5][P]
    const int RS = 5 * a.P;
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
    int F = -1;
    T res = T(0);
    for (int k = 0; k < limit; ++k) {
        if (!trunc && k >= 2) {
            T rr;
            if (!sweep_residual(a, k - 2, rr)) return;
            if (rr < a.tol) {
                F = k - 1;
                res = rr;
                break;
            }
        }
        const T *Ak = (k & 1) ? a.A1 : a.A0;
        T *An = (k & 1) ? a.A0 : a.A1;
        if (k > 0 && !wait_neighbours(a.done, k, &a.work->status, a.spin_limit)) return;
        T local = T(0);
        for (int c0 = r_begin; c0 < r_end; c0 += a.chunk_rows) {
            const int c1 = min(r_end, c0 + a.chunk_rows);
            if (!stage_rows(a, As, Ak, c0, c1, RS, &bar, phase)) return;
            const int ncell = (c1 - c0) * a.P;
            for (int i = threadIdx.x; i < ncell; i += blockDim.x) {
                const int rr = i / a.P, col = i - rr * a.P;
                const int row = c0 + rr;
                const int y = row * a.P + col;
                const unsigned cw = __ldg(a.cell + y);
                T o[5] = {T(0), T(0), T(0), T(0), T(0)};
                const T *rowp = As + (rr + 1) * RS;
                T diff = T(0);
                if (QV_CELL_FREE(cw) && y != a.goal) {
                    diff = fib_cell(a, y, col, cw, rowp, o);
                } else {
#pragma unroll
                    for (int b = 0; b < 5; ++b) {
                        const T dd = fabs(rowp[b * a.P + col]);
                        diff = dd > diff ? dd : diff;
                    }
                }
                T *dst = An + static_cast<size_t>(row) * RS + col;
#pragma unroll
                for (int b = 0; b < 5; ++b) dst[b * a.P] = o[b];
                local = diff > local ? diff : local;
            }
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!trunc || k == limit - 1) {
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
        if (!trunc && limit >= 2) {
            T rr;
            if (!sweep_residual(a, limit - 2, rr)) return;
            if (rr < a.tol) {
                F = limit - 1;
                res = rr;
            }
        }
        if (F < 0) {
            T rr;
            if (!sweep_residual(a, limit - 1, rr)) return;
            F = limit;
            res = rr;
        }
    }
    // alpha_F: this CTA's own rows, written by its own threads in sweep F - 1
    // (no CTA runs sweep F + 1, which would rewrite that buffer)
    __syncthreads();
    const T *Af = (F & 1) ? a.A1 : a.A0;
    const size_t plane = static_cast<size_t>(a.H) * a.P;
    const int n = (r_end - r_begin) * RS;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int rr = i / RS, rem = i - rr * RS;
        const int b = rem / a.P, col = rem - b * a.P;
        const size_t y = static_cast<size_t>(r_begin + rr) * a.P + col;
        const T v = Af[static_cast<size_t>(r_begin) * RS + i];
        a.Q[b * plane + y] = static_cast<float>(v);
        if (a.alpha_out) a.alpha_out[b * plane + y] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.sweeps_out = F;
        *a.residual_out = res;
    }
}

// ---------------------------------------------------------------- temporally blocked sweeps
// The same iteration with s sweeps per exchange, as k_vi_blocked does it for
// the value iteration: CTA i owns rows [i R, i R + R) and stages alpha_{b s}
// (five planes a row) on rows [i R - s, i R + R + s) once per block; sweep j
// of the block covers the owned rows widened by s - 1 - j rows, reading the
// cell words and arrival rewards from shared memory; every sweep's owned
// rows go to plane k mod 2 s of a ring in global memory and its residual to
// a per-block slot; the test of block b runs before block b + 2, so the
// result is exactly the first alpha_{k+1} with max |alpha_{k+1} - alpha_k| <
// tol (or alpha_truncated).
template <typename T>
__global__ void __launch_bounds__(kFIBThreads) k_fib_blocked(FibArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ T s_red[kFIBThreads / 32][kMaxBlock];
    const int s = a.s, R = a.R, P = a.P, H = a.H, RS = 5 * P;
    const int r_begin = static_cast<int>(blockIdx.x) * R, r_end = min(H, r_begin + R);
    const int base = r_begin - s;  // grid row of shared row 0
    const int nrows = R + 2 * s;
    const int glo = max(0, base), ghi = min(H, base + nrows);  // grid rows held
    const size_t nb = static_cast<size_t>(nrows) * RS;
    T *const A0s = reinterpret_cast<T *>(smem_raw), *const A1s = A0s + nb;
    T *const rws = A0s + 2 * nb;  // arrival rewards, [row][P]
    uint16_t *cws = reinterpret_cast<uint16_t *>(rws + static_cast<size_t>(nrows) * P);
    const size_t plane = static_cast<size_t>(H) * RS;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    // cell words (the goal's free bit cleared: it is never updated) and
    // arrival rewards of every row held, once
    for (int i = threadIdx.x; i < (ghi - glo) * P; i += blockDim.x) {
        const int y = glo * P + i;
        const uint16_t cw = __ldg(a.cell + y);
        cws[(glo - base) * P + i] = y == a.goal ? static_cast<uint16_t>(cw & 0x7FFFu) : cw;
        rws[(glo - base) * P + i] = fib_stage_reward(a, y);
    }
    __syncthreads();
    unsigned phase = 0;
    const bool trunc = a.truncated > 0;
    const int limit = trunc ? a.truncated : a.max_sweeps;
    const int nblk = (limit + s - 1) / s;
    int F = -1;
    T res = T(0);
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
        const T *src = b == 0 ? a.A0 : a.hist + static_cast<size_t>(k0 % (2 * s)) * plane;
        if (threadIdx.x == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            fence_proxy_async();
            const unsigned bytes = static_cast<unsigned>((ghi - glo) * RS * sizeof(T));
            mbar_arrive_expect_tx(&bar, bytes);
            bulk_copy_g2s(A0s + (glo - base) * RS, src + static_cast<size_t>(glo) * RS, bytes, &bar);
        }
        const bool ok = mbar_wait_bounded(&bar, phase);
        const int failed = __syncthreads_or(ok ? 0 : 1);
        if (failed) {
            if (threadIdx.x == 0) atomicOr(&a.work->status, kErrTimeout);
            if (!ok) mbar_wait_bounded(&bar, phase);  // let the copy in flight land before leaving
            return;
        }
        phase ^= 1u;
        int cur = 0;
        for (int j = 0; j < ns; ++j) {
            const int k = k0 + j;  // this sweep makes alpha_{k+1}
            const int ext = ns - 1 - j;
            const int lo = max(0, r_begin - ext), hi = min(H, r_end + ext);
            T *dst = a.hist + static_cast<size_t>((k + 1) % (2 * s)) * plane;
            const T *Ac = cur ? A1s : A0s;
            T *An = cur ? A0s : A1s;
            T lm = T(0);
            if (active)
                for (int row = lo + rsub; row < hi; row += rstep) {
                    const bool own = row >= r_begin && row < r_end;
                    const int sr = row - base;
                    for (int col = c0; col < P; col += cstep) {
                        const int t = sr * P + col;
                        const unsigned cw = cws[t];
                        const T *rowp = Ac + static_cast<size_t>(sr) * RS;
                        T o[5] = {T(0), T(0), T(0), T(0), T(0)};
                        T diff = T(0);
                        if (QV_CELL_FREE(cw)) {  // free and not the goal
                            const unsigned blk = QV_CELL_BLOCKED(cw);
                            T al[5][5];
                            unsigned lab[5];
                            T r[5];
#pragma unroll
                            for (int q = 0; q < 5; ++q) al[4][q] = rowp[q * P + col];
                            lab[4] = QV_CELL_LABEL(cw);
                            r[4] = rws[t];
                            const int drow[4] = {-RS, 0, RS, 0};
                            const int dcol[4] = {0, 1, 0, -1};
                            const int dt[4] = {-P, 1, P, -1};
#pragma unroll
                            for (int d = 0; d < 4; ++d) {
                                if (blk & (1u << d)) {
#pragma unroll
                                    for (int q = 0; q < 5; ++q) al[d][q] = al[4][q];
                                    lab[d] = lab[4];
                                    r[d] = r[4];
                                } else {
                                    const T *qp = rowp + drow[d] + col + dcol[d];
#pragma unroll
                                    for (int q = 0; q < 5; ++q) al[d][q] = qp[q * P];
                                    lab[d] = QV_CELL_LABEL(static_cast<unsigned>(cws[t + dt[d]]));
                                    r[d] = rws[t + dt[d]];
                                }
                            }
                            diff = fib_core(a, al, lab, r, o);
                        } else {
#pragma unroll
                            for (int q = 0; q < 5; ++q) {
                                const T dd = fabs(rowp[q * P + col]);
                                diff = dd > diff ? dd : diff;
                            }
                        }
                        T *np_ = An + static_cast<size_t>(sr) * RS + col;
#pragma unroll
                        for (int q = 0; q < 5; ++q) np_[q * P] = o[q];
                        if (own) {
                            lm = diff > lm ? diff : lm;
                            T *gp = dst + static_cast<size_t>(row) * RS + col;
#pragma unroll
                            for (int q = 0; q < 5; ++q) gp[q * P] = o[q];
                        }
                    }
                }
            lm = warp_max(lm);
            if (lane == 0) s_red[wid][j] = lm;
            __syncthreads();
            cur ^= 1;
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (threadIdx.x < ns) {
            T m = T(0);
            for (int w = 0; w < kFIBThreads / 32; ++w) m = s_red[w][threadIdx.x] > m ? s_red[w][threadIdx.x] : m;
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
    // alpha_F on this CTA's own rows (plane F mod 2 s, written by its own
    // threads): Q and the caller's alpha
    __syncthreads();
    const T *Af = a.hist + static_cast<size_t>(F % (2 * s)) * plane;
    const size_t qplane = static_cast<size_t>(H) * P;
    const int n = (r_end - r_begin) * RS;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int rr = i / RS, rem = i - rr * RS;
        const int q = rem / P, col = rem - q * P;
        const size_t y = static_cast<size_t>(r_begin + rr) * P + col;
        const T v = Af[static_cast<size_t>(r_begin) * RS + i];
        a.Q[q * qplane + y] = static_cast<float>(v);
        if (a.alpha_out) a.alpha_out[q * qplane + y] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *a.sweeps_out = F;
        *a.residual_out = res;
    }
}

template <typename T>
size_t fib_ws_bytes(int H, int P, int nslots) {
    size_t b = sizeof(VIWork);
    b = (b + 255) & ~size_t(255);
    b += 2 * static_cast<size_t>(H) * 5 * P * sizeof(T);  // two alpha buffers
    b = (b + 255) & ~size_t(255);
    b += kResRing * nslots * sizeof(T) + sizeof(int) + sizeof(T) + 64;
    b = (b + 255) & ~size_t(255);
    b += nslots * sizeof(unsigned) + 64;  // progress flags, residual arrival counters
    b = (b + 255) & ~size_t(255);
    b += 2 * kMaxBlock * static_cast<size_t>(H) * 5 * P * sizeof(T);  // the blocked sweeps' ring of planes
    b = (b + 255) & ~size_t(255);
    b += static_cast<size_t>(kResRing) * kMaxBlock * nslots * sizeof(T);  // their per-block residuals
    return (b + 255) & ~size_t(255);
}

// Shape of the blocked FIB sweeps (one 512-thread CTA per SM, R rows each,
// s sweeps per exchange) from the same kind of cost model as the value
// iteration's: an exchange of about 4 us shared by s sweeps against the
// R + s - 1 rows a sweep computes on average, each cell's Eq. 7 backup about
// six times a Bellman backup; the one-sweep-per-exchange kernel
// (exchange plus cells per SM) is kept unless the blocked one is predicted
// 10 % faster.  FP32 only (the FP64 backup needs more registers than a
// 512-thread CTA leaves).  QVTS_VI_BLOCK (1, 2, 4, 8; "0") forces s or the
// one-sweep kernel, as for the value iteration.
template <typename T>
bool fib_block_shape(int H, int P, int nsm, int &G, int &R, int &s, int &nh, size_t &smem) {
    if (sizeof(T) != 4) return false;
    R = (H + nsm - 1) / nsm;
    G = (H + R - 1) / R;
    const char *env = std::getenv("QVTS_VI_BLOCK");
    const int forced = env ? std::atoi(env) : 0;
    if (env && *env && forced == 0) return false;
    const double xb = 4000.0, cb = 2.5, ob = 1000.0;  // ns: exchange, per cell computed, fixed
    const double xo = 4300.0, co = 4.6;
    const double t_old = xo + co * static_cast<double>(H) * P / nsm;
    double best = 1e30;
    for (int c : {8, 4, 2, 1}) {
        if (forced > 0 && c != forced) continue;
        const int h = (c + R - 1) / R;
        const size_t sm = static_cast<size_t>(R + 2 * c) * P * (10 * sizeof(T) + sizeof(T) + sizeof(uint16_t));
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
qv_status run_fib(const qv_model_t *m, double tol, int max_sweeps, int truncated, T *d_alpha, float *d_Q,
                  void *d_ws, size_t ws_bytes, int *sweeps_out, double *residual_out, cudaStream_t st) {
    const int H = m->H, P = m->pitch;
    int bG = 0, bR = 0, bs = 0, bnh = 0;
    size_t bsmem = 0;
    bool blocked = fib_block_shape<T>(H, P, qv_num_sms(), bG, bR, bs, bnh, bsmem) && bG <= 1024;
    if (blocked) {
        void *bk = reinterpret_cast<void *>(k_fib_blocked<T>);
        if (qv_check_cuda(cudaFuncSetAttribute(bk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(bsmem)),
                          "smem attr") != QV_OK)
            return QV_ERR_CUDA;
        int per_sm = 0;
        if (qv_check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bk, kFIBThreads, bsmem),
                          "occupancy") != QV_OK)
            return QV_ERR_CUDA;
        blocked = per_sm >= 1 && bG <= per_sm * qv_num_sms();
    }
    const size_t row_bytes = static_cast<size_t>(5) * P * sizeof(T);
    int dev = 0, optin = 0;
    if (qv_check_cuda(cudaGetDevice(&dev), "device") != QV_OK ||
        qv_check_cuda(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attribute") !=
            QV_OK)
        return QV_ERR_CUDA;
    // static shared memory of the kernel (mbarrier, residual scratch) stays below 1 KB
    if (3 * row_bytes + 1024 > static_cast<size_t>(optin))
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: pitch %d too wide to stage three rows of %s alpha",
                            P, sizeof(T) == 8 ? "FP64" : "FP32");
    const size_t budget = std::max<size_t>(40 * 1024, 3 * row_bytes);
    int chunk = static_cast<int>(budget / row_bytes) - 2;
    size_t smem = static_cast<size_t>(chunk + 2) * row_bytes;
    void *kern = reinterpret_cast<void *>(k_fib_iteration<T>);
    if (smem > 40 * 1024 &&
        qv_check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)),
                      "smem attr") != QV_OK)
        return QV_ERR_CUDA;
    int per_sm = 0;
    if (qv_check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem), "occupancy") !=
        QV_OK)
        return QV_ERR_CUDA;
    if (per_sm < 1) return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: kernel does not fit an SM");
    int grid = std::min(per_sm * qv_num_sms(), 1024);
    grid = std::min(grid, H);
    const int rows_per_cta = (H + grid - 1) / grid;
    grid = (H + rows_per_cta - 1) / rows_per_cta;
    chunk = std::min(chunk, rows_per_cta);
    smem = static_cast<size_t>(chunk + 2) * row_bytes;
    if (ws_bytes < fib_ws_bytes<T>(H, P, 1024))
        return qv_set_error(QV_ERR_WORKSPACE, "fib_value_iterate: workspace %zu < %zu bytes", ws_bytes,
                            fib_ws_bytes<T>(H, P, 1024));
    char *ws = static_cast<char *>(d_ws);
    VIWork *work = reinterpret_cast<VIWork *>(ws);
    size_t off = (sizeof(VIWork) + 255) & ~size_t(255);
    T *A0 = reinterpret_cast<T *>(ws + off);
    T *A1 = A0 + static_cast<size_t>(H) * 5 * P;
    off = (off + 2 * static_cast<size_t>(H) * 5 * P * sizeof(T) + 255) & ~size_t(255);
    T *slots = reinterpret_cast<T *>(ws + off);
    int *d_sweeps = reinterpret_cast<int *>(slots + kResRing * 1024);
    T *d_res = reinterpret_cast<T *>(reinterpret_cast<char *>(d_sweeps) + 16);
    const size_t off_flags =
        (off + kResRing * 1024 * sizeof(T) + sizeof(int) + sizeof(T) + 64 + 255) & ~size_t(255);
    unsigned *flags = reinterpret_cast<unsigned *>(ws + off_flags);
    unsigned *arrive = flags + 1024;
    if (qv_check_cuda(cudaMemsetAsync(work, 0, sizeof(VIWork), st), "memset") != QV_OK ||
        qv_check_cuda(cudaMemsetAsync(A0, 0, static_cast<size_t>(H) * 5 * P * sizeof(T), st), "memset") !=
            QV_OK ||
        qv_check_cuda(cudaMemsetAsync(flags, 0, sizeof(unsigned) * (1024 + 16), st), "memset") != QV_OK)
        return QV_ERR_CUDA;
    FibArgs<T> a;
    a.H = H;
    a.W = m->W;
    a.P = P;
    a.cell = m->d_cell;
    a.cost = m->d_cost;
    a.goal = m->goal;
    a.slip = m->slip;
    a.gamma = static_cast<T>(m->discount);
    a.tol = static_cast<T>(tol);
    a.acc = static_cast<T>(m->accuracy);
    a.eta = (T(1) - static_cast<T>(m->accuracy)) / static_cast<T>(m->num_beacons);
    a.nz = m->num_beacons + 1;
    a.max_sweeps = max_sweeps;
    a.truncated = truncated;
    a.A0 = A0;
    a.A1 = A1;
    a.alpha_out = d_alpha;
    a.Q = d_Q;
    a.res_slots = slots;
    a.work = work;
    a.sweeps_out = d_sweeps;
    a.residual_out = d_res;
    a.chunk_rows = chunk;
    a.done = flags;
    a.arrive = arrive;
    a.spin_limit = qv_cross_spin_limit();
    const size_t off_hist = (off_flags + 1024 * sizeof(unsigned) + 64 + 255) & ~size_t(255);
    a.hist = reinterpret_cast<T *>(ws + off_hist);
    const size_t off_bres =
        (off_hist + 2 * kMaxBlock * static_cast<size_t>(H) * 5 * P * sizeof(T) + 255) & ~size_t(255);
    a.bres = reinterpret_cast<T *>(ws + off_bres);
    a.s = bs;
    a.R = bR;
    a.nh = bnh;
    void *args[] = {&a};
    if (blocked) {
        if (qv_check_cuda(cudaLaunchCooperativeKernel(reinterpret_cast<void *>(k_fib_blocked<T>), bG, kFIBThreads,
                                                      args, bsmem, st),
                          "FIB iteration launch") != QV_OK)
            return QV_ERR_CUDA;
    } else if (qv_check_cuda(cudaLaunchCooperativeKernel(kern, grid, 256, args, smem, st), "FIB iteration launch") !=
               QV_OK) {
        return QV_ERR_CUDA;
    }
    VIWork hw;
    int hs = 0;
    T hr = T(0);
    if (qv_check_cuda(cudaMemcpyAsync(&hw, work, sizeof(hw), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&hs, d_sweeps, sizeof(int), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&hr, d_res, sizeof(T), cudaMemcpyDeviceToHost, st), "copy") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "FIB iteration") != QV_OK)
        return QV_ERR_CUDA;
    if (hw.status & kErrTimeout)
        return qv_set_error(QV_ERR_TIMEOUT, "fib_value_iterate: a wait on another CTA or a copy timed out");
    if (sweeps_out) *sweeps_out = hs;
    if (residual_out) *residual_out = static_cast<double>(hr);
    if (truncated <= 0 && !(static_cast<double>(hr) < tol))
        return qv_set_error(QV_ERR_NOT_CONVERGED, "fib_value_iterate: residual %g after %d sweeps",
                            static_cast<double>(hr), hs);
    return QV_OK;
}

}  // namespace qv

extern "C" size_t fib_value_iterate_workspace_bytes(const qv_model_t *m, int32_t dtype) {
    if (!m) return 0;
    return dtype == QV_F64 ? qv::fib_ws_bytes<double>(m->H, m->pitch, 1024)
                           : qv::fib_ws_bytes<float>(m->H, m->pitch, 1024);
}

extern "C" qv_status fib_value_iterate(const qv_model_t *m, int32_t dtype, double tol, int32_t max_sweeps,
                                       int32_t truncated, void *d_alpha, float *d_Q, void *d_ws, size_t ws_bytes,
                                       int32_t *sweeps_out, double *residual_out, qv_stream_t stream) {
    QV_RANGE("fib_value_iterate");
    if (const qv_status inj = qv_injected_fault("fib_value_iterate", true)) return inj;
    if (!m || !m->d_cell || !d_Q || !d_ws)
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: null pointer");
    if (m->H < 1 || m->W < 1 || m->pitch != QV_PITCH(m->W) || m->W > QV_MAX_WIDTH)
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: bad grid");
    if (!(m->discount > 0.0f && m->discount < 1.0f) || !(m->slip >= 0.0f && m->slip <= 0.5f))
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: discount or slip out of range");
    if (m->num_beacons < 1 || m->num_beacons > QV_MAX_BEACONS || !(m->accuracy > 0.0f && m->accuracy <= 1.0f))
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: beacons or accuracy out of range");
    if (truncated <= 0 && max_sweeps < 1)
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: max_sweeps < 1");
    if ((reinterpret_cast<uintptr_t>(d_ws) | reinterpret_cast<uintptr_t>(d_alpha)) & 15)
        return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: buffers must be 16-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dtype == QV_F64)
        return qv::run_fib<double>(m, tol, max_sweeps, truncated, static_cast<double *>(d_alpha), d_Q, d_ws,
                                   ws_bytes, sweeps_out, residual_out, st);
    if (dtype == QV_F32)
        return qv::run_fib<float>(m, tol, max_sweeps, truncated, static_cast<float *>(d_alpha), d_Q, d_ws,
                                  ws_bytes, sweeps_out, residual_out, st);
    return qv_set_error(QV_ERR_INVALID, "fib_value_iterate: dtype %d", dtype);
}
