// qv_tree.cu -- level-synchronous QV-tree expansion, leaves and backup.
//
// Kernels per tree level l (all episodes of a batch in one launch each):
//   k_stats   one pass over every V-node belief of level l (Alg. 2: every
//             action): the motion stencil for all five actions (Eq. 3
//             numerator, Eq. 10), the label histograms that give P(z | b, a)
//             (Eq. 3 denominator), R(b, a) (Sec. III), K Philox draws per
//             action inverted through the CDF (Alg. 3-4), the unique samples
//             with their frequencies.  At the deepest internal level of the
//             fused leaf mode it also accumulates Q-weighted histograms so
//             every leaf value max_a' sum_y b'(y) Q(a', y) (Eq. 4, Alg. 5)
//             follows without writing the leaf beliefs.
//   k_compact prefix sum of the unique-sample counts: the children of level
//             l+1 in (parent, action, z) order.
//   k_update  Phi(b, a, z) of Eq. 3 for every child: one read of the parent
//             band, one coalesced write per child.
//   k_leaf    (materialised leaves) streams leaf beliefs against Q.
//   k_backup  Alg. 6 / 7 bottom-up and the root argmax.
//
// Persistent kernels walk a flat list of (episode, node, band-range) work
// items whose per-level prefix sums live on the device, so one launch covers
// episodes of uneven size and the host never waits for a level's size.
#include <cstdio>
#include <cstring>
#include <vector>

#include "qv_common.cuh"

namespace qv {

constexpr int kMaxD = QV_MAX_DEPTH;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLeafGroup = 4;
constexpr int kBandCells = 4096;
constexpr float kBoundaryEps = 1e-6f;

struct EpDev {
    int H, W, P, N;          // N = H * P
    int B, goal;
    float slip, acc, eta, gamma;
    const uint16_t *cell;
    const float *cost;
    const float *Q;          // [5][N]
    const float *b0;         // [N]
    int band_rows, bands;
    uint32_t episode;
    int cap[kMaxD + 1];      // node capacity of each level
    int node_base[kMaxD + 1];   // gid of local node 0 of level l
    int inode_base[kMaxD + 1];  // iid of local node 0 of internal level l < d
    int items[kMaxD + 1];    // stats work items per node at level l
    int uitems[kMaxD + 1];   // update work items per node at level l
    long long part_base[kMaxD + 1];   // partial record index of local node 0 (items > 1)
    long long belief_off[kMaxD + 1];  // float offset of level-l beliefs (level 0: b0)
};

struct ResultDev {
    int action;
    float value;
    float q[5];
    int pad;
};

struct PlanDev {
    int E, depth, K, weight_mode, leaf_mode, Bmax, rec_len;
    uint64_t seed;
    const EpDev *eps;
    float *beliefs;
    int *count;        // [(d+1)][E]
    int *wb_stats;     // [(d+1)][E+1]
    int *wb_upd;       // [(d+1)][E+1]
    int *wb_leaf;      // [E+1]
    // per node (gid over every level)
    int *parent, *action, *obs;
    float *weight, *pz, *value;
    unsigned long long *code;
    // per internal node (iid over levels < d)
    unsigned *counter;
    float *R, *UQ;     // [iid][5]
    int *nchild, *choff;
    int *samples;      // [iid][5][K]
    int *slot_z, *slot_cnt;
    float *slot_P, *slot_w, *slot_val;
    float *partials;
    unsigned *status;
    unsigned long long *boundary;
    unsigned *ep_done; // [d+1]
    ResultDev *result; // [E]
    const int *replay;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ int find_episode(const int *wb, int E, int w) {
    int lo = 0, hi = E - 1;  // last e with wb[e] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldcg(wb + mid) <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ const float *node_belief(const PlanDev &pl, const EpDev &ep, int l, int local) {
    if (l == 0) return ep.b0;
    return pl.beliefs + ep.belief_off[l] + static_cast<long long>(local) * ep.N;
}

__device__ __forceinline__ void fill_self_lut(float *lut, float slip) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) lut[i] = self_weight(i >> 4, i & 15, slip);
}

// Stage grid rows [r0-1, r1+1) of belief `b` into smem rows 0..(r1-r0+1);
// rows outside the grid are zero.  One bulk (TMA) copy; bounded wait.
__device__ bool stage_band(const EpDev &ep, const float *b, int r0, int r1, float *sb, uint64_t *bar,
                           unsigned &phase, unsigned *status) {
    const int P = ep.P;
    __syncthreads();  // previous readers of sb are done
    if (r0 == 0)
        for (int i = threadIdx.x; i < P; i += blockDim.x) sb[i] = 0.0f;
    if (r1 == ep.H)
        for (int i = threadIdx.x; i < P; i += blockDim.x) sb[(r1 - r0 + 1) * P + i] = 0.0f;
    fence_proxy_async();
    __syncthreads();
    const int lo = max(0, r0 - 1), hi = min(ep.H, r1 + 1);
    if (threadIdx.x == 0) {
        const unsigned bytes = static_cast<unsigned>((hi - lo) * P * sizeof(float));
        mbar_arrive_expect_tx(bar, bytes);
        bulk_copy_g2s(sb + (lo - (r0 - 1)) * P, b + static_cast<size_t>(lo) * P, bytes, bar);
    }
    const bool ok = mbar_wait_bounded(bar, phase);
    // one decision for the whole CTA, so an early exit never splits it
    const int failed = __syncthreads_or(ok ? 0 : 1);
    if (failed) {
        if (threadIdx.x == 0) atomicOr(status, kErrTimeout);
        if (!ok) mbar_wait_bounded(bar, phase);  // let the copy in flight land before leaving
    }
    phase ^= 1u;
    return failed == 0;
}

// Predicted mass of the 4 cells of group (rr, col) of a staged band.
struct Group4 {
    float out[4][5];
    unsigned cw[4];
};
__device__ __forceinline__ void predict_group(const EpDev &ep, const float *sb, int rr, int col, int y,
                                              const float *lut, Group4 &g) {
    const int P = ep.P;
    const float4 up = *reinterpret_cast<const float4 *>(sb + rr * P + col);
    const float4 mid = *reinterpret_cast<const float4 *>(sb + (rr + 1) * P + col);
    const float4 dn = *reinterpret_cast<const float4 *>(sb + (rr + 2) * P + col);
    const float left = col > 0 ? sb[(rr + 1) * P + col - 1] : 0.0f;
    const float right = col + 4 < P ? sb[(rr + 1) * P + col + 4] : 0.0f;
    const ushort4 cw4 = __ldg(reinterpret_cast<const ushort4 *>(ep.cell + y));
    const float u[4] = {up.x, up.y, up.z, up.w};
    const float m[6] = {left, mid.x, mid.y, mid.z, mid.w, right};
    const float d[4] = {dn.x, dn.y, dn.z, dn.w};
    const unsigned cws[4] = {cw4.x, cw4.y, cw4.z, cw4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned cw = cws[j];
        const unsigned in = QV_CELL_INFLOW(cw);
        float nb[4];
        nb[kDirN] = (in & 1u) ? u[j] : 0.0f;
        nb[kDirE] = (in & 2u) ? m[j + 2] : 0.0f;
        nb[kDirS] = (in & 4u) ? d[j] : 0.0f;
        nb[kDirW] = (in & 8u) ? m[j] : 0.0f;
        predict_cell(nb, m[j + 1], cw, (y + j) == ep.goal, ep.slip, lut, g.out[j]);
        g.cw[j] = cw;
    }
}

// ---------------------------------------------------------------- init
__global__ void k_init(PlanDev pl, int n_counter) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = tid; i < n_counter; i += gridDim.x * blockDim.x) pl.counter[i] = 0u;
    for (int e = tid; e < pl.E; e += gridDim.x * blockDim.x) {
        pl.count[e] = 1;
        const EpDev &ep = pl.eps[e];
        const int g = ep.node_base[0];
        pl.parent[g] = -1;
        pl.action[g] = -1;
        pl.obs[g] = -1;
        pl.weight[g] = 1.0f;
        pl.pz[g] = 1.0f;
        pl.code[g] = 0ull;
    }
    if (tid == 0) {
        *pl.status = 0u;
        *pl.boundary = 0ull;
        for (int l = 0; l <= pl.depth; ++l) pl.ep_done[l] = 0u;
    }
}

// ---------------------------------------------------------------- stats + sampling
struct StatsSmem {
    float *sb;      // band buffer
    float *hist;    // [5][Bmax] label mass (z < B)
    float *histq;   // [5][Bmax][5] Q-weighted label mass (fused leaves)
    float *tot;     // [35]: null mass [5], reward sums [5], Q-weighted null [25]
    float *red;     // [kWarps][35]
    float *P;       // [5][Bmax+1]
    float *C;       // [5][Bmax+1]
    int *cnt;       // [5][Bmax+1]
    float *T;       // [25]
    float *lut;     // [64]
};

__device__ void finalize_node(const PlanDev &pl, const EpDev &ep, int l, int local, bool fused,
                              StatsSmem &s) {
    const int B = ep.B, nz = B + 1, K = pl.K;
    const int iid = ep.inode_base[l] + local;
    const int gid = ep.node_base[l] + local;
    const float eta = ep.eta, acc = ep.acc;
    for (int i = threadIdx.x; i < 5 * nz; i += blockDim.x) s.cnt[i] = 0;
    if (fused && threadIdx.x < 25) {
        const int a = threadIdx.x / 5, ap = threadIdx.x % 5;
        float t = s.tot[10 + threadIdx.x];
        for (int z = 0; z < B; ++z) t += s.histq[(a * pl.Bmax + z) * 5 + ap];
        s.T[threadIdx.x] = t;
    }
    if (threadIdx.x < 5) {
        const int a = threadIdx.x;
        float S = s.tot[a];
        for (int z = 0; z < B; ++z) S += s.hist[a * pl.Bmax + z];
        float run = 0.0f;
        for (int z = 0; z < nz; ++z) {
            const float M = z < B ? s.hist[a * pl.Bmax + z] : s.tot[a];
            const float p = fmaf(acc - eta, M, eta * S);
            s.P[a * nz + z] = p;
            run = run + p;
            s.C[a * nz + z] = run;
        }
        const float bg = __ldg(node_belief(pl, ep, l, local) + ep.goal);
        pl.R[iid * 5 + a] = s.tot[5 + a] - 100.0f * bg;
    }
    __syncthreads();
    const unsigned long long code = pl.code[gid];
    for (int t = threadIdx.x; t < 5 * K; t += blockDim.x) {
        const int a = t / K, k = t - a * K;
        const float *C = s.C + a * nz;
        const float u = sample_uniform(pl.seed, ep.episode, l, code * 5ull + a, k);
        int z;
        if (pl.replay) {
            z = pl.replay[(static_cast<long long>(iid) * 5 + a) * K + k];
            z = min(max(z, 0), B);
        } else {
            const float t_u = u * C[B];
            int lo = 0, hi = B;  // first z with t_u < C[z]
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (t_u < C[mid]) hi = mid;
                else lo = mid + 1;
            }
            z = lo;
        }
        const float inv = 1.0f / C[B];
        const bool near = (z < B && fabsf(u - C[z] * inv) < kBoundaryEps) ||
                          (z > 0 && fabsf(u - C[z - 1] * inv) < kBoundaryEps);
        if (near) atomicAdd(pl.boundary, 1ull);
        pl.samples[(static_cast<long long>(iid) * 5 + a) * K + k] = z;
        atomicAdd(&s.cnt[a * nz + z], 1);
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        const int a = threadIdx.x;
        const long long sb = (static_cast<long long>(iid) * 5 + a) * K;
        int m = 0;
        float psum = 0.0f;
        for (int z = 0; z < nz; ++z) {
            const int c = s.cnt[a * nz + z];
            if (!c) continue;
            const float p = s.P[a * nz + z];
            pl.slot_z[sb + m] = z;
            pl.slot_cnt[sb + m] = c;
            pl.slot_P[sb + m] = p;
            psum += p;
            if (fused) {
                float best = -3.402823466e38f;
                for (int ap = 0; ap < 5; ++ap) {
                    const float mq = z < B ? s.histq[(a * pl.Bmax + z) * 5 + ap] : s.tot[10 + a * 5 + ap];
                    const float v = fmaf(acc - eta, mq, eta * s.T[a * 5 + ap]) / p;
                    best = v > best ? v : best;
                }
                pl.slot_val[sb + m] = best;
            }
            ++m;
        }
        for (int j = 0; j < m; ++j)
            pl.slot_w[sb + j] = pl.weight_mode == QV_WEIGHT_MARGINAL ? pl.slot_P[sb + j] / psum
                                                                      : static_cast<float>(pl.slot_cnt[sb + j]) / K;
        pl.nchild[iid * 5 + a] = m;
    }
}

template <bool FUSED>
__global__ void __launch_bounds__(kThreads) k_stats(PlanDev pl, int l, int band_floats) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_last;
    const int Bm = pl.Bmax;
    StatsSmem s;
    float *f = reinterpret_cast<float *>(smem_raw);
    s.sb = f;
    f += band_floats;
    s.hist = f;
    f += 5 * Bm;
    s.histq = f;
    f += FUSED ? 25 * Bm : 0;
    s.tot = f;
    f += 36;
    s.red = f;
    f += kWarps * 36;
    s.P = f;
    f += 5 * (Bm + 1);
    s.C = f;
    f += 5 * (Bm + 1);
    s.cnt = reinterpret_cast<int *>(f);
    f += 5 * (Bm + 1);
    s.T = f;
    f += 28;
    s.lut = f;
    constexpr int NV = FUSED ? 35 : 10;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const int *wb = pl.wb_stats + l * (pl.E + 1);
    const int total = __ldcg(wb + pl.E);
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int e = find_episode(wb, pl.E, w);
        const EpDev &ep = pl.eps[e];
        const int items = ep.items[l];
        const int rel = w - __ldcg(wb + e);
        const int local = rel / items, item = rel - local * items;
        const int B = ep.B;
        const float *b = node_belief(pl, ep, l, local);
        __syncthreads();
        fill_self_lut(s.lut, ep.slip);
        for (int i = threadIdx.x; i < 5 * Bm; i += blockDim.x) s.hist[i] = 0.0f;
        if (FUSED)
            for (int i = threadIdx.x; i < 25 * Bm; i += blockDim.x) s.histq[i] = 0.0f;
        float acc_null[5], acc_r[5], acc_q[FUSED ? 25 : 1];
#pragma unroll
        for (int a = 0; a < 5; ++a) acc_null[a] = acc_r[a] = 0.0f;
#pragma unroll
        for (int i = 0; i < (FUSED ? 25 : 1); ++i) acc_q[i] = 0.0f;
        const int band0 = static_cast<int>((static_cast<long long>(item) * ep.bands) / items);
        const int band1 = static_cast<int>((static_cast<long long>(item + 1) * ep.bands) / items);
        const int P4 = ep.P >> 2;
        const size_t plane = static_cast<size_t>(ep.N);
        for (int band = band0; band < band1; ++band) {
            const int r0 = band * ep.band_rows, r1 = min(ep.H, r0 + ep.band_rows);
            if (!stage_band(ep, b, r0, r1, s.sb, &bar, phase, pl.status)) return;
            const int ng = (r1 - r0) * P4;
            for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
                const int rr = gi / P4, col = (gi - rr * P4) << 2;
                const int y = (r0 + rr) * ep.P + col;
                Group4 g;
                predict_group(ep, s.sb, rr, col, y, s.lut, g);
                float4 q4[5];
                if (FUSED) {
#pragma unroll
                    for (int ap = 0; ap < 5; ++ap) q4[ap] = __ldg(reinterpret_cast<const float4 *>(ep.Q + ap * plane + y));
                }
                float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ep.cost) c4 = __ldg(reinterpret_cast<const float4 *>(ep.cost + y));
                const float cst[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const unsigned cw = g.cw[j];
                    const int lab = QV_CELL_LABEL(cw);
                    const float r = stage_reward(QV_CELL_FREE(cw), (y + j) == ep.goal, cst[j]);
                    float qj[5];
                    if (FUSED) {
                        qj[0] = (&q4[0].x)[j];
                        qj[1] = (&q4[1].x)[j];
                        qj[2] = (&q4[2].x)[j];
                        qj[3] = (&q4[3].x)[j];
                        qj[4] = (&q4[4].x)[j];
                    }
                    if (lab >= B) {
#pragma unroll
                        for (int a = 0; a < 5; ++a) {
                            const float v = g.out[j][a];
                            acc_null[a] += v;
                            acc_r[a] = fmaf(v, r, acc_r[a]);
                            if (FUSED) {
#pragma unroll
                                for (int ap = 0; ap < 5; ++ap) acc_q[a * 5 + ap] = fmaf(v, qj[ap], acc_q[a * 5 + ap]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int a = 0; a < 5; ++a) {
                            const float v = g.out[j][a];
                            acc_r[a] = fmaf(v, r, acc_r[a]);
                            if (v != 0.0f) {
                                atomicAdd(&s.hist[a * Bm + lab], v);
                                if (FUSED) {
#pragma unroll
                                    for (int ap = 0; ap < 5; ++ap) atomicAdd(&s.histq[(a * Bm + lab) * 5 + ap], v * qj[ap]);
                                }
                            }
                        }
                    }
                }
            }
        }
        // block reduction of the register accumulators into s.tot
        {
            float vals[NV];
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                vals[a] = acc_null[a];
                vals[5 + a] = acc_r[a];
            }
            if constexpr (FUSED) {
#pragma unroll
                for (int i = 0; i < 25; ++i) vals[10 + i] = acc_q[i];
            }
            const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                const float v = warp_sum(vals[i]);
                if (lane == 0) s.red[wid * 36 + i] = v;
            }
            __syncthreads();
            if (threadIdx.x < NV) {
                float t = 0.0f;
                for (int k = 0; k < kWarps; ++k) t += s.red[k * 36 + threadIdx.x];
                s.tot[threadIdx.x] = t;
            }
            __syncthreads();
        }
        const int iid = ep.inode_base[l] + local;
        if (items > 1) {
            // partial record: [hist 5B][histq 25B][tot NV]
            float *rec = pl.partials + (ep.part_base[l] + static_cast<long long>(local) * items + item) * pl.rec_len;
            for (int i = threadIdx.x; i < 5 * B; i += blockDim.x) rec[i] = s.hist[(i / B) * Bm + (i % B)];
            if (FUSED)
                for (int i = threadIdx.x; i < 25 * B; i += blockDim.x)
                    rec[5 * B + i] = s.histq[((i / 5) / B * Bm + (i / 5) % B) * 5 + i % 5];
            for (int i = threadIdx.x; i < NV; i += blockDim.x) rec[(FUSED ? 30 : 5) * B + i] = s.tot[i];
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned prev = atomicAdd(pl.counter + iid, 1u);
                s_last = (prev == static_cast<unsigned>(items - 1)) ? 1 : 0;
                if (s_last) pl.counter[iid] = 0u;
            }
            __syncthreads();
            if (!s_last) continue;
            __threadfence();
            // the last item sums every record in item order
            const float *base = pl.partials + (ep.part_base[l] + static_cast<long long>(local) * items) * pl.rec_len;
            for (int i = threadIdx.x; i < 5 * B; i += blockDim.x) {
                float t = 0.0f;
                for (int it = 0; it < items; ++it) t += __ldcg(base + static_cast<long long>(it) * pl.rec_len + i);
                s.hist[(i / B) * Bm + (i % B)] = t;
            }
            if (FUSED)
                for (int i = threadIdx.x; i < 25 * B; i += blockDim.x) {
                    float t = 0.0f;
                    for (int it = 0; it < items; ++it)
                        t += __ldcg(base + static_cast<long long>(it) * pl.rec_len + 5 * B + i);
                    s.histq[((i / 5) / B * Bm + (i / 5) % B) * 5 + i % 5] = t;
                }
            for (int i = threadIdx.x; i < NV; i += blockDim.x) {
                float t = 0.0f;
                for (int it = 0; it < items; ++it)
                    t += __ldcg(base + static_cast<long long>(it) * pl.rec_len + (FUSED ? 30 : 5) * B + i);
                s.tot[i] = t;
            }
            __syncthreads();
        }
        finalize_node(pl, ep, l, local, FUSED, s);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- compaction
__device__ int block_exclusive_scan(int v, int *s_warp, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int k = 0; k < kWarps; ++k) {
            const int t = s_warp[k];
            s_warp[k] = run;
            run += t;
        }
        s_warp[kWarps] = run;
    }
    __syncthreads();
    const int ex = x - v + s_warp[wid];
    total = s_warp[kWarps];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(kThreads) k_compact(PlanDev pl, int l, int fused_leaf) {
    __shared__ int s_warp[kWarps + 1];
    __shared__ int s_last;
    const int e = blockIdx.x;
    const EpDev &ep = pl.eps[e];
    const int n = __ldcg(pl.count + l * pl.E + e);
    const int M = n * 5;
    const long long ia = static_cast<long long>(ep.inode_base[l]) * 5;
    int running = 0;
    for (int base = 0; base < M; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < M ? pl.nchild[ia + i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, s_warp, total);
        if (i < M) pl.choff[ia + i] = running + ex;
        running += total;
    }
    int nn = running;
    if (nn > ep.cap[l + 1]) {
        if (threadIdx.x == 0) atomicOr(pl.status, kErrCapacity);
        nn = ep.cap[l + 1];
    }
    if (threadIdx.x == 0) pl.count[(l + 1) * pl.E + e] = nn;
    const int K = pl.K, nz = ep.B + 1;
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        const int node = i / 5, a = i - node * 5;
        const int m = pl.nchild[ia + i];
        const int off = pl.choff[ia + i];
        const long long sb = (ia + i) * K;
        const unsigned long long pcode = pl.code[ep.node_base[l] + node];
        for (int j = 0; j < m; ++j) {
            const int c = off + j;
            if (c >= nn) break;
            const int g = ep.node_base[l + 1] + c;
            const int z = pl.slot_z[sb + j];
            pl.parent[g] = node;
            pl.action[g] = a;
            pl.obs[g] = z;
            pl.weight[g] = pl.slot_w[sb + j];
            pl.pz[g] = pl.slot_P[sb + j];
            pl.code[g] = (pcode * 5ull + a) * static_cast<unsigned long long>(nz) + z;
            if (fused_leaf) pl.value[g] = pl.slot_val[sb + j];
        }
    }
    // the last episode to finish publishes the work-list prefixes of level l+1
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(pl.ep_done + l, 1u) == static_cast<unsigned>(pl.E - 1)) ? 1 : 0;
    __syncthreads();
    if (!s_last || threadIdx.x != 0) return;
    __threadfence();
    pl.ep_done[l] = 0u;
    const int l1 = l + 1;
    int ws = 0, wu = 0, wl = 0;
    for (int k = 0; k < pl.E; ++k) {
        const int c = __ldcg(pl.count + l1 * pl.E + k);
        const EpDev &q = pl.eps[k];
        pl.wb_stats[l1 * (pl.E + 1) + k] = ws;
        pl.wb_upd[l1 * (pl.E + 1) + k] = wu;
        if (l1 == pl.depth) pl.wb_leaf[k] = wl;
        if (l1 < pl.depth) {
            ws += c * q.items[l1];
            wu += c * q.uitems[l1];
        }
        wl += (c + kLeafGroup - 1) / kLeafGroup;
    }
    pl.wb_stats[l1 * (pl.E + 1) + pl.E] = ws;
    pl.wb_upd[l1 * (pl.E + 1) + pl.E] = wu;
    if (l1 == pl.depth) pl.wb_leaf[pl.E] = wl;
}

// ---------------------------------------------------------------- belief update (Eq. 3)
__global__ void __launch_bounds__(kThreads) k_update(PlanDev pl, int l, int band_floats) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_n[5], s_off[5];
    __shared__ int s_z[5 * QV_MAX_K];
    __shared__ float s_sa[5 * QV_MAX_K], s_se[5 * QV_MAX_K];
    __shared__ float s_lut[64];
    float *sb = reinterpret_cast<float *>(smem_raw);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const int K = pl.K;
    const int *wb = pl.wb_upd + l * (pl.E + 1);
    const int total = __ldcg(wb + pl.E);
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int e = find_episode(wb, pl.E, w);
        const EpDev &ep = pl.eps[e];
        const int items = ep.uitems[l];
        const int rel = w - __ldcg(wb + e);
        const int local = rel / items, item = rel - local * items;
        const long long ia = static_cast<long long>(ep.inode_base[l] + local) * 5;
        __syncthreads();
        fill_self_lut(s_lut, ep.slip);
        if (threadIdx.x < 5) {
            s_n[threadIdx.x] = pl.nchild[ia + threadIdx.x];
            s_off[threadIdx.x] = pl.choff[ia + threadIdx.x];
        }
        for (int t = threadIdx.x; t < 5 * K; t += blockDim.x) {
            const int a = t / K, j = t - a * K;
            const long long sbi = (ia + a) * K + j;
            const float p = pl.slot_P[sbi];
            s_z[t] = pl.slot_z[sbi];
            s_sa[t] = ep.acc / p;
            s_se[t] = ep.eta / p;
        }
        const float *b = node_belief(pl, ep, l, local);
        float *child0 = pl.beliefs + ep.belief_off[l + 1];
        const int cap = ep.cap[l + 1];
        const int band0 = static_cast<int>((static_cast<long long>(item) * ep.bands) / items);
        const int band1 = static_cast<int>((static_cast<long long>(item + 1) * ep.bands) / items);
        const int P4 = ep.P >> 2;
        for (int band = band0; band < band1; ++band) {
            const int r0 = band * ep.band_rows, r1 = min(ep.H, r0 + ep.band_rows);
            if (!stage_band(ep, b, r0, r1, sb, &bar, phase, pl.status)) return;
            const int ng = (r1 - r0) * P4;
            for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
                const int rr = gi / P4, col = (gi - rr * P4) << 2;
                const int y = (r0 + rr) * ep.P + col;
                Group4 g;
                predict_group(ep, sb, rr, col, y, s_lut, g);
                int lab[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) lab[j] = QV_CELL_LABEL(g.cw[j]);
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    const int n = s_n[a], off = s_off[a];
                    for (int m = 0; m < n; ++m) {
                        const int c = off + m;
                        if (c >= cap) break;
                        const int t = a * K + m;
                        const int z = s_z[t];
                        const float sa = s_sa[t], se = s_se[t];
                        float4 o;
                        o.x = g.out[0][a] * (lab[0] == z ? sa : se);
                        o.y = g.out[1][a] * (lab[1] == z ? sa : se);
                        o.z = g.out[2][a] * (lab[2] == z ? sa : se);
                        o.w = g.out[3][a] * (lab[3] == z ? sa : se);
                        *reinterpret_cast<float4 *>(child0 + static_cast<long long>(c) * ep.N + y) = o;
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- leaf values (Eq. 4)
__device__ __forceinline__ float4 ld_stream(const float *p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__global__ void __launch_bounds__(kThreads) k_leaf(PlanDev pl, int l) {
    __shared__ float s_red[kWarps][kLeafGroup * 5];
    const int *wb = pl.wb_leaf;
    const int total = __ldcg(wb + pl.E);
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int e = find_episode(wb, pl.E, w);
        const EpDev &ep = pl.eps[e];
        const int n = __ldcg(pl.count + l * pl.E + e);
        const int first = (w - __ldcg(wb + e)) * kLeafGroup;
        const int cnt = min(kLeafGroup, n - first);
        float acc[kLeafGroup][5];
#pragma unroll
        for (int i = 0; i < kLeafGroup; ++i)
#pragma unroll
            for (int a = 0; a < 5; ++a) acc[i][a] = 0.0f;
        const size_t plane = static_cast<size_t>(ep.N);
        const int n4 = ep.N >> 2;
        for (int i4 = threadIdx.x; i4 < n4; i4 += blockDim.x) {
            float4 q[5];
#pragma unroll
            for (int a = 0; a < 5; ++a) q[a] = __ldg(reinterpret_cast<const float4 *>(ep.Q + a * plane) + i4);
#pragma unroll
            for (int i = 0; i < kLeafGroup; ++i) {
                if (i < cnt) {
                    const float4 b = ld_stream(node_belief(pl, ep, l, first + i) + 4 * i4);
#pragma unroll
                    for (int a = 0; a < 5; ++a)
                        acc[i][a] = fmaf(b.x, q[a].x, fmaf(b.y, q[a].y, fmaf(b.z, q[a].z, fmaf(b.w, q[a].w, acc[i][a]))));
                }
            }
        }
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kLeafGroup; ++i)
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                const float v = warp_sum(acc[i][a]);
                if (lane == 0) s_red[wid][i * 5 + a] = v;
            }
        __syncthreads();
        if (threadIdx.x < cnt) {
            const int i = threadIdx.x;
            float sums[5];
            float best = -3.402823466e38f;
            int ba = 0;
            for (int a = 0; a < 5; ++a) {
                float t = 0.0f;
                for (int k = 0; k < kWarps; ++k) t += s_red[k][i * 5 + a];
                sums[a] = t;
                if (t > best) {
                    best = t;
                    ba = a;
                }
            }
            pl.value[ep.node_base[l] + first + i] = best;
            if (l == 0) {  // depth-0 plan: the root is the leaf
                ResultDev r;
                r.action = ba;
                r.value = best;
                for (int a = 0; a < 5; ++a) r.q[a] = sums[a];
                r.pad = 0;
                pl.result[e] = r;
            }
        }
    }
}

// ---------------------------------------------------------------- backup (Alg. 6, 7)
__global__ void __launch_bounds__(kThreads) k_backup(PlanDev pl) {
    const int e = blockIdx.x;
    const EpDev &ep = pl.eps[e];
    for (int l = pl.depth - 1; l >= 0; --l) {
        const int n = __ldcg(pl.count + l * pl.E + e);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const long long ia = static_cast<long long>(ep.inode_base[l] + i) * 5;
            float best = -3.402823466e38f;
            for (int a = 0; a < 5; ++a) {
                const int m = pl.nchild[ia + a], off = pl.choff[ia + a];
                float s = 0.0f;
                for (int j = 0; j < m; ++j) {
                    const int g = ep.node_base[l + 1] + off + j;
                    s = fmaf(pl.weight[g], pl.value[g], s);
                }
                const float uq = fmaf(ep.gamma, s, pl.R[ia + a]);
                pl.UQ[ia + a] = uq;
                best = uq > best ? uq : best;
            }
            pl.value[ep.node_base[l] + i] = best;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long ia = static_cast<long long>(ep.inode_base[0]) * 5;
        ResultDev r;
        r.action = 0;
        for (int a = 0; a < 5; ++a) {
            r.q[a] = pl.UQ[ia + a];
            if (r.q[a] > r.q[r.action]) r.action = a;
        }
        r.value = pl.value[ep.node_base[0]];
        r.pad = 0;
        pl.result[e] = r;
    }
}

}  // namespace qv

// ======================================================================== host side
struct qv_plan {
    int E = 0;
    qv_plan_params_t params{};
    std::vector<qv::EpDev> eps;
    qv::PlanDev dev{};
    char *ws = nullptr;
    size_t bytes = 0;
    int n_counter = 0;
    int grid_stats[QV_MAX_DEPTH + 1] = {};
    int grid_upd[QV_MAX_DEPTH + 1] = {};
    int grid_leaf = 0;
    int band_floats = 0;
    size_t smem_stats = 0, smem_stats_fused = 0, smem_upd = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

struct Layout {
    size_t total = 0;
    size_t off_eps, off_count, off_wbs, off_wbu, off_wbl, off_parent, off_action, off_obs, off_weight, off_pz,
        off_value, off_code, off_counter, off_R, off_UQ, off_nchild, off_choff, off_samples, off_slot_z,
        off_slot_cnt, off_slot_P, off_slot_w, off_slot_val, off_partials, off_status, off_boundary, off_ep_done,
        off_result, off_beliefs;
    long long NT = 0, NI = 0, n_part = 0, n_belief = 0;
    int Bmax = 1, rec_len = 0, band_floats = 0;
    std::vector<qv::EpDev> eps;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

qv_status validate(int E, const qv_model_t *models, const qv_plan_params_t *p) {
    if (E < 1) return qv_set_error(QV_ERR_INVALID, "plan: E=%d", E);
    if (!models || !p) return qv_set_error(QV_ERR_INVALID, "plan: null pointer");
    if (p->depth < 0 || p->depth > QV_MAX_DEPTH) return qv_set_error(QV_ERR_INVALID, "plan: depth %d", p->depth);
    if (p->K < 1 || p->K > QV_MAX_K) return qv_set_error(QV_ERR_INVALID, "plan: K %d", p->K);
    if (p->weight_mode != QV_WEIGHT_FREQ && p->weight_mode != QV_WEIGHT_MARGINAL)
        return qv_set_error(QV_ERR_INVALID, "plan: weight_mode %d", p->weight_mode);
    if (p->leaf_mode != QV_LEAF_FUSED && p->leaf_mode != QV_LEAF_MATERIALISE)
        return qv_set_error(QV_ERR_INVALID, "plan: leaf_mode %d", p->leaf_mode);
    if (p->d_replay && E != 1) return qv_set_error(QV_ERR_INVALID, "plan: replay needs E = 1");
    for (int e = 0; e < E; ++e) {
        const qv_model_t &m = models[e];
        if (!m.d_cell) return qv_set_error(QV_ERR_INVALID, "plan: episode %d has no cell words", e);
        if (m.H < 1 || m.W < 1 || m.W > QV_MAX_WIDTH || m.pitch != ((m.W + 3) / 4) * 4)
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d grid %dx%d pitch %d", e, m.H, m.W, m.pitch);
        if (m.num_beacons < 1 || m.num_beacons > QV_MAX_BEACONS)
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d B=%d", e, m.num_beacons);
        if (m.goal < 0 || m.goal >= m.H * m.pitch || m.goal % m.pitch >= m.W)
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d goal %d", e, m.goal);
        if (!(m.slip >= 0.f && m.slip <= 0.5f) || !(m.accuracy > 0.f && m.accuracy <= 1.f) ||
            !(m.discount > 0.f && m.discount < 1.f))
            return qv_set_error(QV_ERR_INVALID, "plan: episode %d slip/accuracy/discount out of range", e);
        // path code: (5 (B+1))^d * 5 must fit below 2^56 for the Philox counter
        double code = 5.0;
        for (int l = 0; l < p->depth; ++l) code *= 5.0 * (m.num_beacons + 1);
        if (code >= 72057594037927936.0)
            return qv_set_error(QV_ERR_INVALID, "plan: depth %d with B=%d overflows the path code", p->depth,
                                m.num_beacons);
    }
    return QV_OK;
}

qv_status make_layout(int E, const qv_model_t *models, const qv_plan_params_t *p, Layout &L) {
    qv_status st = validate(E, models, p);
    if (st != QV_OK) return st;
    const int D = p->depth, K = p->K;
    const int nsm = qv_num_sms();
    const long long target = 8LL * nsm;
    L.eps.assign(E, qv::EpDev{});
    L.Bmax = 1;
    for (int e = 0; e < E; ++e) L.Bmax = std::max(L.Bmax, models[e].num_beacons);
    // level capacities and bases
    long long NB[QV_MAX_DEPTH + 1] = {};
    for (int e = 0; e < E; ++e) {
        const qv_model_t &m = models[e];
        qv::EpDev &ep = L.eps[e];
        ep.H = m.H;
        ep.W = m.W;
        ep.P = m.pitch;
        ep.N = m.H * m.pitch;
        ep.B = m.num_beacons;
        ep.goal = m.goal;
        ep.slip = m.slip;
        ep.acc = m.accuracy;
        ep.eta = (1.0f - m.accuracy) / static_cast<float>(m.num_beacons);
        ep.gamma = m.discount;
        ep.cell = m.d_cell;
        ep.cost = m.d_cost;
        ep.episode = p->episode + static_cast<uint32_t>(e);
        ep.band_rows = std::max(1, std::min(m.H, qv::kBandCells / m.pitch));
        ep.bands = (m.H + ep.band_rows - 1) / ep.band_rows;
        const long long br = std::min<long long>(K, m.num_beacons + 1) * 5;
        long long c = 1;
        for (int l = 0; l <= D; ++l) {
            if (c > (1LL << 30)) return qv_set_error(QV_ERR_INVALID, "plan: level %d capacity overflow", l);
            ep.cap[l] = static_cast<int>(c);
            NB[l] += c;
            c *= br;
        }
        L.band_floats = std::max(L.band_floats, (ep.band_rows + 2) * ep.P);
    }
    // global id bases (levels concatenated, episodes concatenated per level)
    long long gbase = 0, ibase = 0;
    long long run_g[QV_MAX_DEPTH + 1], run_i[QV_MAX_DEPTH + 1];
    for (int l = 0; l <= D; ++l) {
        run_g[l] = gbase;
        gbase += NB[l];
        if (l < D) {
            run_i[l] = ibase;
            ibase += NB[l];
        }
    }
    L.NT = gbase;
    L.NI = std::max<long long>(ibase, 1);
    if (L.NT > (1LL << 31) - 1 || L.NI * 5 * K > (1LL << 40))
        return qv_set_error(QV_ERR_INVALID, "plan: tree too large");
    L.n_part = 0;
    L.n_belief = 0;
    const bool mat = p->leaf_mode == QV_LEAF_MATERIALISE || D == 0;
    for (int l = 0; l <= D; ++l) {
        const long long items = std::max<long long>(1, (target + NB[l] - 1) / std::max<long long>(NB[l], 1));
        for (int e = 0; e < E; ++e) {
            qv::EpDev &ep = L.eps[e];
            ep.node_base[l] = static_cast<int>(run_g[l]);
            run_g[l] += ep.cap[l];
            ep.items[l] = static_cast<int>(std::min<long long>(items, ep.bands));
            ep.uitems[l] = ep.items[l];
            if (l < D) {
                ep.inode_base[l] = static_cast<int>(run_i[l]);
                run_i[l] += ep.cap[l];
                if (ep.items[l] > 1) {
                    ep.part_base[l] = L.n_part;
                    L.n_part += static_cast<long long>(ep.cap[l]) * ep.items[l];
                } else {
                    ep.part_base[l] = -1;
                }
            } else {
                ep.inode_base[l] = -1;
                ep.part_base[l] = -1;
            }
            const bool store = (l >= 1) && (l < D || (l == D && mat));
            if (store) {
                ep.belief_off[l] = L.n_belief;
                L.n_belief += static_cast<long long>(ep.cap[l]) * ep.N;
            } else {
                ep.belief_off[l] = -1;
            }
        }
    }
    L.rec_len = 30 * L.Bmax + 36;
    // byte layout
    size_t o = 0;
    auto take = [&](size_t bytes) {
        o = align_up(o, 256);
        const size_t r = o;
        o += bytes;
        return r;
    };
    L.off_eps = take(sizeof(qv::EpDev) * E);
    L.off_count = take(sizeof(int) * (D + 1) * E);
    L.off_wbs = take(sizeof(int) * (D + 1) * (E + 1));
    L.off_wbu = take(sizeof(int) * (D + 1) * (E + 1));
    L.off_wbl = take(sizeof(int) * (E + 1));
    L.off_parent = take(sizeof(int) * L.NT);
    L.off_action = take(sizeof(int) * L.NT);
    L.off_obs = take(sizeof(int) * L.NT);
    L.off_weight = take(sizeof(float) * L.NT);
    L.off_pz = take(sizeof(float) * L.NT);
    L.off_value = take(sizeof(float) * L.NT);
    L.off_code = take(sizeof(unsigned long long) * L.NT);
    L.off_counter = take(sizeof(unsigned) * L.NI);
    L.off_R = take(sizeof(float) * L.NI * 5);
    L.off_UQ = take(sizeof(float) * L.NI * 5);
    L.off_nchild = take(sizeof(int) * L.NI * 5);
    L.off_choff = take(sizeof(int) * L.NI * 5);
    L.off_samples = take(sizeof(int) * L.NI * 5 * K);
    L.off_slot_z = take(sizeof(int) * L.NI * 5 * K);
    L.off_slot_cnt = take(sizeof(int) * L.NI * 5 * K);
    L.off_slot_P = take(sizeof(float) * L.NI * 5 * K);
    L.off_slot_w = take(sizeof(float) * L.NI * 5 * K);
    L.off_slot_val = take(sizeof(float) * L.NI * 5 * K);
    L.off_partials = take(sizeof(float) * std::max<long long>(L.n_part, 1) * L.rec_len);
    L.off_status = take(sizeof(unsigned));
    L.off_boundary = take(sizeof(unsigned long long));
    L.off_ep_done = take(sizeof(unsigned) * (D + 1));
    L.off_result = take(sizeof(qv::ResultDev) * E);
    L.off_beliefs = take(sizeof(float) * std::max<long long>(L.n_belief, 4));
    L.total = align_up(o, 256);
    return QV_OK;
}

template <typename T>
T *at(char *ws, size_t off) {
    return reinterpret_cast<T *>(ws + off);
}

int occupancy_grid(const void *fn, size_t smem, long long max_work) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, qv::kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long g = std::min<long long>(std::max<long long>(max_work, 1), static_cast<long long>(per_sm) * qv_num_sms());
    return static_cast<int>(g);
}

qv_status launch_all(qv_plan_t *pl, cudaStream_t st) {
    const qv::PlanDev &d = pl->dev;
    const int D = pl->params.depth;
    const int E = pl->E;
    const int ninit = static_cast<int>(std::min<long long>((pl->n_counter + 255) / 256 + 1, 4LL * qv_num_sms()));
    qv::k_init<<<ninit, 256, 0, st>>>(d, pl->n_counter);
    for (int l = 0; l < D; ++l) {
        const bool fused = (l == D - 1) && pl->params.leaf_mode == QV_LEAF_FUSED;
        if (fused)
            qv::k_stats<true><<<pl->grid_stats[l], qv::kThreads, pl->smem_stats_fused, st>>>(d, l, pl->band_floats);
        else
            qv::k_stats<false><<<pl->grid_stats[l], qv::kThreads, pl->smem_stats, st>>>(d, l, pl->band_floats);
        qv::k_compact<<<E, qv::kThreads, 0, st>>>(d, l, fused ? 1 : 0);
        if (!fused) qv::k_update<<<pl->grid_upd[l], qv::kThreads, pl->smem_upd, st>>>(d, l, pl->band_floats);
    }
    if (D == 0 || pl->params.leaf_mode == QV_LEAF_MATERIALISE) qv::k_leaf<<<pl->grid_leaf, qv::kThreads, 0, st>>>(d, D);
    if (D > 0) qv::k_backup<<<E, qv::kThreads, 0, st>>>(d);
    return qv_check_cuda(cudaGetLastError(), "qv_plan_run launch");
}

}  // namespace

extern "C" size_t qv_plan_workspace_bytes(int32_t E, const qv_model_t *models, const qv_plan_params_t *params) {
    Layout L;
    if (make_layout(E, models, params, L) != QV_OK) return 0;
    return L.total;
}

extern "C" qv_status qv_plan_create(int32_t E, const qv_model_t *models, const float *const *d_Q,
                                    const float *const *d_b0, const qv_plan_params_t *params, void *d_ws,
                                    size_t ws_bytes, qv_plan_t **plan_out, qv_stream_t stream) {
    if (!plan_out || !d_Q || !d_b0 || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv_plan_create: null pointer");
    *plan_out = nullptr;
    Layout L;
    qv_status st = make_layout(E, models, params, L);
    if (st != QV_OK) return st;
    if (ws_bytes < L.total)
        return qv_set_error(QV_ERR_WORKSPACE, "qv_plan_create: workspace %zu < %zu bytes", ws_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_create: workspace must be 256-byte aligned");
    for (int e = 0; e < E; ++e) {
        if (!d_Q[e] || !d_b0[e]) return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d null Q/b0", e);
        if ((reinterpret_cast<uintptr_t>(d_Q[e]) | reinterpret_cast<uintptr_t>(d_b0[e])) & 15)
            return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d Q/b0 not 16-byte aligned", e);
        if (models[e].d_cost && (reinterpret_cast<uintptr_t>(models[e].d_cost) & 15))
            return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d cost not 16-byte aligned", e);
        if (reinterpret_cast<uintptr_t>(models[e].d_cell) & 7)
            return qv_set_error(QV_ERR_INVALID, "qv_plan_create: episode %d cell words not 8-byte aligned", e);
        L.eps[e].Q = d_Q[e];
        L.eps[e].b0 = d_b0[e];
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    qv_plan_t *pl = new qv_plan_t;
    pl->E = E;
    pl->params = *params;
    pl->eps = L.eps;
    pl->ws = static_cast<char *>(d_ws);
    pl->bytes = L.total;
    pl->n_counter = static_cast<int>(L.NI);
    pl->band_floats = L.band_floats;
    char *ws = pl->ws;
    qv::PlanDev &d = pl->dev;
    d.E = E;
    d.depth = params->depth;
    d.K = params->K;
    d.weight_mode = params->weight_mode;
    d.leaf_mode = params->leaf_mode;
    d.Bmax = L.Bmax;
    d.rec_len = L.rec_len;
    d.seed = params->seed;
    d.eps = at<qv::EpDev>(ws, L.off_eps);
    d.beliefs = at<float>(ws, L.off_beliefs);
    d.count = at<int>(ws, L.off_count);
    d.wb_stats = at<int>(ws, L.off_wbs);
    d.wb_upd = at<int>(ws, L.off_wbu);
    d.wb_leaf = at<int>(ws, L.off_wbl);
    d.parent = at<int>(ws, L.off_parent);
    d.action = at<int>(ws, L.off_action);
    d.obs = at<int>(ws, L.off_obs);
    d.weight = at<float>(ws, L.off_weight);
    d.pz = at<float>(ws, L.off_pz);
    d.value = at<float>(ws, L.off_value);
    d.code = at<unsigned long long>(ws, L.off_code);
    d.counter = at<unsigned>(ws, L.off_counter);
    d.R = at<float>(ws, L.off_R);
    d.UQ = at<float>(ws, L.off_UQ);
    d.nchild = at<int>(ws, L.off_nchild);
    d.choff = at<int>(ws, L.off_choff);
    d.samples = at<int>(ws, L.off_samples);
    d.slot_z = at<int>(ws, L.off_slot_z);
    d.slot_cnt = at<int>(ws, L.off_slot_cnt);
    d.slot_P = at<float>(ws, L.off_slot_P);
    d.slot_w = at<float>(ws, L.off_slot_w);
    d.slot_val = at<float>(ws, L.off_slot_val);
    d.partials = at<float>(ws, L.off_partials);
    d.status = at<unsigned>(ws, L.off_status);
    d.boundary = at<unsigned long long>(ws, L.off_boundary);
    d.ep_done = at<unsigned>(ws, L.off_ep_done);
    d.result = at<qv::ResultDev>(ws, L.off_result);
    d.replay = params->d_replay;
    // static level-0 work prefixes; every other level is written on the device
    const int D = params->depth;
    std::vector<int> wbs((D + 1) * (E + 1), 0), wbu((D + 1) * (E + 1), 0), wbl(E + 1, 0);
    int s0 = 0, u0 = 0, l0 = 0;
    for (int e = 0; e < E; ++e) {
        wbs[e] = s0;
        wbu[e] = u0;
        s0 += D > 0 ? L.eps[e].items[0] : 0;
        u0 += D > 0 ? L.eps[e].uitems[0] : 0;
        wbl[e] = l0;
        l0 += 1;
    }
    wbs[E] = s0;
    wbu[E] = u0;
    wbl[E] = l0;
    if (qv_check_cuda(cudaMemcpyAsync(const_cast<qv::EpDev *>(d.eps), L.eps.data(), sizeof(qv::EpDev) * E,
                                      cudaMemcpyHostToDevice, cs),
                      "descriptor upload") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(d.wb_stats, wbs.data(), sizeof(int) * wbs.size(), cudaMemcpyHostToDevice, cs),
                      "descriptor upload") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(d.wb_upd, wbu.data(), sizeof(int) * wbu.size(), cudaMemcpyHostToDevice, cs),
                      "descriptor upload") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(d.wb_leaf, wbl.data(), sizeof(int) * wbl.size(), cudaMemcpyHostToDevice, cs),
                      "descriptor upload") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(cs), "descriptor upload") != QV_OK) {
        delete pl;
        return QV_ERR_CUDA;
    }
    // launch shapes
    const int Bm = L.Bmax;
    const size_t fixed = sizeof(float) * (5 * Bm + 36 + qv::kWarps * 36 + 15 * (Bm + 1) + 28 + 64);
    pl->smem_stats = sizeof(float) * L.band_floats + fixed;
    pl->smem_stats_fused = pl->smem_stats + sizeof(float) * 25 * Bm;
    pl->smem_upd = sizeof(float) * L.band_floats;
    {
        if (qv_check_cuda(cudaFuncSetAttribute(qv::k_stats<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(pl->smem_stats_fused)),
                          "smem attr") != QV_OK ||
            qv_check_cuda(cudaFuncSetAttribute(qv::k_stats<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(pl->smem_stats)),
                          "smem attr") != QV_OK ||
            qv_check_cuda(cudaFuncSetAttribute(qv::k_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(pl->smem_upd)),
                          "smem attr") != QV_OK) {
            delete pl;
            return QV_ERR_CUDA;
        }
    }
    for (int l = 0; l <= D; ++l) {
        long long ws_items = 0, wu_items = 0;
        for (int e = 0; e < E; ++e) {
            ws_items += static_cast<long long>(L.eps[e].cap[l]) * L.eps[e].items[l];
            wu_items += static_cast<long long>(L.eps[e].cap[l]) * L.eps[e].uitems[l];
        }
        const bool fused = (l == D - 1) && params->leaf_mode == QV_LEAF_FUSED;
        pl->grid_stats[l] = fused ? occupancy_grid(reinterpret_cast<const void *>(qv::k_stats<true>),
                                                   pl->smem_stats_fused, ws_items)
                                  : occupancy_grid(reinterpret_cast<const void *>(qv::k_stats<false>), pl->smem_stats,
                                                   ws_items);
        pl->grid_upd[l] = occupancy_grid(reinterpret_cast<const void *>(qv::k_update), pl->smem_upd, wu_items);
    }
    long long leaf_items = 0;
    for (int e = 0; e < E; ++e) leaf_items += (L.eps[e].cap[D] + qv::kLeafGroup - 1) / qv::kLeafGroup;
    pl->grid_leaf = occupancy_grid(reinterpret_cast<const void *>(qv::k_leaf), 0, leaf_items);
    *plan_out = pl;
    return QV_OK;
}

extern "C" qv_status qv_plan_run(qv_plan_t *pl, qv_stream_t stream) {
    if (!pl) return qv_set_error(QV_ERR_INVALID, "qv_plan_run: null plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (pl->graph) return qv_check_cuda(cudaGraphLaunch(pl->graph, st), "qv_plan_run graph launch");
    return launch_all(pl, st);
}

extern "C" qv_status qv_plan_capture_graph(qv_plan_t *pl, qv_stream_t stream) {
    if (!pl) return qv_set_error(QV_ERR_INVALID, "qv_plan_capture_graph: null plan");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st == nullptr) return qv_set_error(QV_ERR_INVALID, "qv_plan_capture_graph: needs a non-default stream");
    if (pl->graph) {
        cudaGraphExecDestroy(pl->graph);
        pl->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (qv_check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture") != QV_OK)
        return QV_ERR_CUDA;
    const qv_status ls = launch_all(pl, st);
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (ls != QV_OK) {
        if (g) cudaGraphDestroy(g);
        return ls;
    }
    if (qv_check_cuda(ce, "end capture") != QV_OK) return QV_ERR_CUDA;
    const cudaError_t ie = cudaGraphInstantiate(&pl->graph, g, 0);
    cudaGraphDestroy(g);
    return qv_check_cuda(ie, "graph instantiate");
}

extern "C" qv_status qv_plan_read(qv_plan_t *pl, qv_plan_result_t *h, qv_stream_t stream) {
    if (!pl || !h) return qv_set_error(QV_ERR_INVALID, "qv_plan_read: null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int E = pl->E, D = pl->params.depth;
    std::vector<qv::ResultDev> r(E);
    std::vector<int> cnt((D + 1) * E);
    unsigned status = 0;
    unsigned long long bnd = 0;
    if (qv_check_cuda(cudaMemcpyAsync(r.data(), pl->dev.result, sizeof(qv::ResultDev) * E, cudaMemcpyDeviceToHost, st),
                      "read results") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(cnt.data(), pl->dev.count, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, st),
                      "read counts") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&status, pl->dev.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                      "read status") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&bnd, pl->dev.boundary, sizeof(bnd), cudaMemcpyDeviceToHost, st),
                      "read boundary") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "qv_plan_read") != QV_OK)
        return QV_ERR_CUDA;
    for (int e = 0; e < E; ++e) {
        qv_plan_result_t &o = h[e];
        std::memset(&o, 0, sizeof(o));
        o.action = r[e].action;
        o.value = r[e].value;
        for (int a = 0; a < 5; ++a) o.q[a] = r[e].q[a];
        for (int l = 0; l <= D; ++l) o.nodes_per_level[l] = cnt[l * E + e];
        o.boundary_samples = static_cast<int64_t>(bnd);
    }
    if (status & qv::kErrTimeout) return qv_set_error(QV_ERR_TIMEOUT, "qv_plan: a bounded device wait timed out");
    if (status & qv::kErrCapacity) return qv_set_error(QV_ERR_CAPACITY, "qv_plan: a level outgrew its capacity");
    return QV_OK;
}

extern "C" void qv_plan_destroy(qv_plan_t *pl) {
    if (!pl) return;
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    delete pl;
}

extern "C" qv_status qv_plan_level(const qv_plan_t *pl, int32_t e, int32_t l, qv_level_view_t *v) {
    if (!pl || !v) return qv_set_error(QV_ERR_INVALID, "qv_plan_level: null pointer");
    if (e < 0 || e >= pl->E || l < 0 || l > pl->params.depth)
        return qv_set_error(QV_ERR_INVALID, "qv_plan_level: episode %d level %d out of range", e, l);
    const qv::EpDev &ep = pl->eps[e];
    const qv::PlanDev &d = pl->dev;
    const int K = pl->params.K;
    std::memset(v, 0, sizeof(*v));
    v->cap = ep.cap[l];
    v->d_count = d.count + l * pl->E + e;
    const int g = ep.node_base[l];
    v->d_parent = d.parent + g;
    v->d_action = d.action + g;
    v->d_obs = d.obs + g;
    v->d_weight = d.weight + g;
    v->d_pz = d.pz + g;
    v->d_value = d.value + g;
    if (l < pl->params.depth) {
        const long long i = ep.inode_base[l];
        v->d_R = d.R + i * 5;
        v->d_UQ = d.UQ + i * 5;
        v->d_nchild = d.nchild + i * 5;
        v->d_samples = d.samples + i * 5 * K;
    }
    if (l == 0) v->d_belief = ep.b0;
    else if (ep.belief_off[l] >= 0) v->d_belief = d.beliefs + ep.belief_off[l];
    return QV_OK;
}

extern "C" qv_status qv_tree_plan_batched(int32_t E, const qv_model_t *models, const float *const *d_Q,
                                          const float *const *d_b0, const qv_plan_params_t *params, void *d_ws,
                                          size_t ws_bytes, qv_plan_result_t *h_results, qv_stream_t stream) {
    qv_plan_t *pl = nullptr;
    qv_status st = qv_plan_create(E, models, d_Q, d_b0, params, d_ws, ws_bytes, &pl, stream);
    if (st != QV_OK) return st;
    st = qv_plan_run(pl, stream);
    if (st == QV_OK) st = qv_plan_read(pl, h_results, stream);
    qv_plan_destroy(pl);
    return st;
}

extern "C" qv_status qv_tree_plan(const qv_model_t *model, const float *d_Q, const float *d_b0,
                                  const qv_plan_params_t *params, void *d_ws, size_t ws_bytes,
                                  qv_plan_result_t *h_result, qv_stream_t stream) {
    return qv_tree_plan_batched(1, model, &d_Q, &d_b0, params, d_ws, ws_bytes, h_result, stream);
}
