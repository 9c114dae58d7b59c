// qv_model9.cu -- the paper's experimental model (Sec. V) on GB300: nine
// actions with 45-degree slips, four occupancy sensors (|Z| = 16), the
// paper's stage reward; MDP value iteration for its Q and the sampled tree of
// Alg. 2-7 on it.
//
// Layout: unpadded row-major [H][W] grids.  Cell word (uint16 per cell):
//   bit t (t = 0..8, t != 4): the neighbour N_t is occupied or outside
//   bit 4: the cell itself is occupied
//   bit 9: the cell is the goal
// The sensors read bits 1, 3, 5, 7 (N_1 up, N_3 left, N_5 right, N_7 down),
// so a cell's sensor pattern p is those four bits, and O(y, z) depends on y
// only through p: O(p, z) = prod_j (p_j == z_j ? p_sensor : 1 - p_sensor).
//
// Expansion of a V-node b for action a needs, per pattern p, the predicted
// mass M[p] = sum over cells of pattern p of bbar_a (then P(z) = sum_p
// O(p, z) M[p], Eq. 3), and at the deepest level the Q-weighted masses
// H[p][a'] = sum over those cells of bbar_a(y) Q(a', y), so that a leaf
// child's value (Eq. 4 with Gamma = {Q(., a')}) is max_a' sum_p O(p, z)
// H[p][a'] / P(z) with no leaf belief written.  The cells are visited in
// pattern order (each pattern's run padded to a whole warp), so every warp
// batch holds one pattern and the sums build up in registers, warp by warp,
// in a fixed order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "qv_common.cuh"
#include "qv_plan_types.cuh"  // kBoundaryEps, the window of a boundary draw

struct qv9;

namespace qv {
namespace {

constexpr int kA9 = QV9_NUM_ACTIONS, kZ9 = QV9_NUM_OBS;
constexpr int kRec9 = kZ9 + kZ9 * kA9 + 1;  // M[16], H[16][9], R
constexpr int kRun9 = 32;                    // pattern runs padded to whole warps
constexpr int kChunk9 = 8192;                // positions per expansion CTA at the deepest level
constexpr int kChunkSmall9 = 1024;           // ... at the levels above it (few nodes, more CTAs)
constexpr int kT9 = 256;                     // threads of the grid kernels
constexpr int kW9 = kT9 / 32;
constexpr int kBand9 = 4096;                 // cells per child-belief CTA
constexpr int kVIResCap = 1 << 17;           // sweeps whose residual is kept

// Move directions clockwise from straight up (1, 2, 5, 8, 7, 6, 3, 0); a
// 45-degree slip of action a moves one step along this ring.  Written as
// functions so that they fold when a is known at compile time.
__host__ __device__ constexpr int ring_at(int i) {
    return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 5 : i == 3 ? 8 : i == 4 ? 7 : i == 5 ? 6 : i == 6 ? 3 : 0;
}
__host__ __device__ constexpr int ring_pos(int a) {
    return a == 1 ? 0 : a == 2 ? 1 : a == 5 ? 2 : a == 8 ? 3 : a == 7 ? 4 : a == 6 ? 5 : a == 3 ? 6 : a == 0 ? 7 : -1;
}

struct M9 {
    int H, W, n, goal;
    float eps, ps, gamma;
    const uint16_t *cw;
};

__device__ __forceinline__ void slips9(int a, int &s1, int &s2) {
    const int i = ring_pos(a);
    s1 = ring_at((i + 1) & 7);
    s2 = ring_at((i + 7) & 7);
}
__device__ __forceinline__ int step9(const M9 &m, int t) { return (t / 3 - 1) * m.W + (t % 3 - 1); }
__device__ __forceinline__ bool occ9(unsigned cw) { return (cw >> 4) & 1u; }
__device__ __forceinline__ int pattern9(unsigned cw) {
    return ((cw >> 1) & 1u) | (((cw >> 3) & 1u) << 1) | (((cw >> 5) & 1u) << 2) | (((cw >> 7) & 1u) << 3);
}
__device__ __forceinline__ float olik9(float ps, int p, int z) {
    float v = 1.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) v *= (((p ^ z) >> j) & 1) ? 1.0f - ps : ps;
    return v;
}

// R(x, a): -2 for stay off the goal, else sum_t r(N_t) T'(x, a, N_t) over
// the move and its two slips, r = -2 on a blocked cell, 0 at the goal, -1
// elsewhere; 0 at the goal and on occupied cells.
template <typename T>
__device__ __forceinline__ T reward9(const M9 &m, int x, unsigned cw, int a) {
    if (occ9(cw) || x == m.goal) return T(0);
    if (a == 4) return T(-2);
    int s1, s2;
    slips9(a, s1, s2);
    auto r = [&](int t) -> T {
        if ((cw >> t) & 1u) return T(-2);
        return x + step9(m, t) == m.goal ? T(0) : T(-1);
    };
    const T w0 = T(1) - T(2) * T(m.eps), w1 = T(m.eps);
    return w0 * r(a) + w1 * r(s1) + w1 * r(s2);
}

// Predicted mass bbar_a(y) = sum_x T(x, a, y) b(x) at a cell y with word cw:
// inflow from the free, non-goal cells x = y - step(t) for t the move and its
// slips, plus y's own mass that stays (the blocked parts of its moves; all
// of it at the goal and for stay).
__device__ __forceinline__ float predict9(const M9 &m, const float *__restrict__ b, int y, unsigned cw, int a) {
    if (occ9(cw)) return 0.0f;
    const float self = __ldg(b + y);
    if (a == 4) return self;
    int s1, s2;
    slips9(a, s1, s2);
    auto in = [&](int t) -> float {
        const int u = 8 - t;  // N_u(y) = y - step(t)
        if ((cw >> u) & 1u) return 0.0f;
        const int x = y + step9(m, u);
        return x == m.goal ? 0.0f : __ldg(b + x);
    };
    const float w0 = 1.0f - 2.0f * m.eps, w1 = m.eps;
    const float v = fmaf(w0, in(a), w1 * (in(s1) + in(s2)));
    if (y == m.goal) return v + self;
    const float stay = w0 * static_cast<float>((cw >> a) & 1u) +
                       w1 * static_cast<float>(((cw >> s1) & 1u) + ((cw >> s2) & 1u));
    return fmaf(stay, self, v);
}

// ---------------------------------------------------------------- value iteration
// One Jacobi sweep k (Vin -> Vout) with its max-abs change added into
// res[k] (FP64 bits; non-negative doubles order like their bit patterns).
// A sweep whose predecessor already met tol does nothing and records the
// sweep count, so the iteration stops at exactly that sweep.
template <typename T>
__global__ void __launch_bounds__(kT9) k9_vi_sweep(M9 m, const T *__restrict__ Vin, T *__restrict__ Vout, int k,
                                                  double tol, unsigned long long *res, int *done, int *nsweeps) {
    __shared__ double s_max[kW9];
    if (*reinterpret_cast<volatile int *>(done)) return;
    if (k > 0 && __longlong_as_double(static_cast<long long>(res[k - 1])) < tol) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *done = 1;
            *nsweeps = k;
        }
        return;
    }
    double dmax = 0.0;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < m.n; x += gridDim.x * blockDim.x) {
        const unsigned cw = m.cw[x];
        T out = T(0);
        if (!occ9(cw) && x != m.goal) {
            T best = T(0);
            for (int a = 0; a < kA9; ++a) {
                T s;
                if (a == 4) {
                    s = Vin[x];
                } else {
                    int s1, s2;
                    slips9(a, s1, s2);
                    auto v = [&](int t) -> T { return ((cw >> t) & 1u) ? Vin[x] : Vin[x + step9(m, t)]; };
                    const T w0 = T(1) - T(2) * T(m.eps), w1 = T(m.eps);
                    s = w0 * v(a) + w1 * v(s1) + w1 * v(s2);
                }
                const T q = reward9<T>(m, x, cw, a) + T(m.gamma) * s;
                best = (a == 0 || q > best) ? q : best;
            }
            out = best;
        }
        Vout[x] = out;
        dmax = fmax(dmax, fabs(static_cast<double>(out) - static_cast<double>(Vin[x])));
    }
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = dmax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = s_max[0];
        for (int w = 1; w < kW9; ++w) b = fmax(b, s_max[w]);
        atomicMax(res + k, static_cast<unsigned long long>(__double_as_longlong(b)));
    }
}

// Q(a, x) = R(x, a) + gamma sum_y T(x, a, y) V(y) in FP32, and V copied out.
template <typename T>
__global__ void __launch_bounds__(kT9) k9_vi_q(M9 m, const T *__restrict__ V, T *__restrict__ Vout,
                                              float *__restrict__ Q) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < m.n; x += gridDim.x * blockDim.x) {
        const unsigned cw = m.cw[x];
        Vout[x] = V[x];
        const bool absorbing = occ9(cw) || x == m.goal;
        for (int a = 0; a < kA9; ++a) {
            T s;
            if (a == 4 || absorbing) {
                s = V[x];
            } else {
                int s1, s2;
                slips9(a, s1, s2);
                auto v = [&](int t) -> T { return ((cw >> t) & 1u) ? V[x] : V[x + step9(m, t)]; };
                const T w0 = T(1) - T(2) * T(m.eps), w1 = T(m.eps);
                s = w0 * v(a) + w1 * v(s1) + w1 * v(s2);
            }
            Q[static_cast<size_t>(a) * m.n + x] = static_cast<float>(reward9<T>(m, x, cw, a) + T(m.gamma) * s);
        }
    }
}

// R(x, a) for every cell and action, FP32 [9][H][W]: a model constant the
// expansion reads instead of recomputing it per cell.
__global__ void __launch_bounds__(kT9) k9_reward_table(M9 m, float *__restrict__ Rt) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < m.n; x += gridDim.x * blockDim.x) {
        const unsigned cw = m.cw[x];
        for (int a = 0; a < kA9; ++a) Rt[static_cast<size_t>(a) * m.n + x] = reward9<float>(m, x, cw, a);
    }
}

// ---------------------------------------------------------------- the tree
struct Lvl9 {  // one level's node arrays
    int *parent, *action, *obs;
    float *weight, *pz, *value;
    unsigned long long *code;
};

// The root: b0 without its occupied cells, and the root's node record.
__global__ void __launch_bounds__(kT9) k9_root(M9 m, const float *__restrict__ b0, float *__restrict__ bel,
                                              Lvl9 L, unsigned long long *bcount) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < m.n; x += gridDim.x * blockDim.x)
        bel[x] = occ9(m.cw[x]) ? 0.0f : b0[x];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        L.parent[0] = -1;
        L.action[0] = -1;
        L.obs[0] = -1;
        L.weight[0] = 1.0f;
        L.pz[0] = 1.0f;
        L.value[0] = 0.0f;
        L.code[0] = 0ull;
        *bcount = 0ull;
    }
}

// Grid (chunks, nodes): the chunk's positions of the pattern order for node
// i and every action at once (the cell's 3x3 neighbourhood, and at the
// deepest level its nine Q values, are loaded once for the nine actions).
// Per action a, M_a[p], the chunk's share of R(b, a) = sum_x b(x) R(x, a)
// (R from the model's table) and at the deepest level the 81 sums
// H_a[p][a'] of bbar_a(y) Q(a', y) build up in registers over a warp's
// batches of one pattern and are reduced over the warp (reduce-scatters of
// 32 values) when the pattern's run ends.  Warps keep their own bins; the
// CTA adds the warps in order into the chunk's record [9][kRec9].
// (Reducing the 81 products of every batch instead, to hold fewer
// registers, was 4 % slower.)
template <bool LEAF>
__global__ void __launch_bounds__(kT9, LEAF ? 1 : 2) k9_expand(M9 m, const float *__restrict__ bel,
                                                              const int *__restrict__ perm,
                                                              const uint16_t *__restrict__ cwp,
                                                              const signed char *__restrict__ bpat, int Kp, int clen,
                                                              int nchunk, const float *__restrict__ Q,
                                                              const float *__restrict__ Rt, float *__restrict__ rec) {
    constexpr int NH = LEAF ? kA9 * kA9 : 1;
    constexpr int NV = kA9 + (LEAF ? kA9 * kA9 : 0);  // values reduced when a pattern's run ends
    __shared__ float bins[kW9][kA9][kRec9];
    const int c = blockIdx.x, i = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float *b = bel + static_cast<size_t>(i) * m.n;
    for (int t = threadIdx.x; t < kW9 * kA9 * kRec9; t += blockDim.x) (&bins[0][0][0])[t] = 0.0f;
    __syncthreads();
    const int k0 = c * clen, k1 = min(Kp, k0 + clen);
    const int nb = (k1 - k0) / 32;
    const int b0 = (nb * w) / kW9, b1 = (nb * (w + 1)) / kW9;
    int cur = -1;
    float accM[kA9], accR[kA9], accH[NH];
#pragma unroll
    for (int a = 0; a < kA9; ++a) accM[a] = accR[a] = 0.0f;
#pragma unroll
    for (int j = 0; j < NH; ++j) accH[j] = 0.0f;
    auto flush = [&]() {
        if (cur < 0) return;
        // values: M_0..M_8, then H_a[.][a'] at 9 + a * 9 + a'
#pragma unroll
        for (int g0 = 0; g0 < NV; g0 += 32) {
            float v[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const int idx = g0 + t;
                v[t] = idx < kA9 ? accM[idx < kA9 ? idx : 0] : (idx < NV ? accH[idx - kA9 < NH ? idx - kA9 : 0] : 0.0f);
            }
            warp_reduce_scatter32(v);
            const int idx = g0 + lane;
            if (idx < kA9) bins[w][idx][cur] += v[0];
            else if (idx < NV) {
                const int a = (idx - kA9) / kA9, j = (idx - kA9) - a * kA9;
                bins[w][a][kZ9 + cur * kA9 + j] += v[0];
            }
        }
#pragma unroll
        for (int a = 0; a < kA9; ++a) accM[a] = 0.0f;
#pragma unroll
        for (int j = 0; j < NH; ++j) accH[j] = 0.0f;
    };
    const float w0 = 1.0f - 2.0f * m.eps, w1 = m.eps;
    // the cell index, cell word and pattern of the next batch are loaded
    // while this batch is computed (they head the chain of dependent loads)
    int y_next = b0 < b1 ? __ldg(perm + k0 + b0 * 32 + lane) : -1;
    unsigned cw_next = b0 < b1 ? __ldg(cwp + k0 + b0 * 32 + lane) : 0u;
    int p_next = b0 < b1 ? bpat[k0 / 32 + b0] : 0;
    for (int bt = b0; bt < b1; ++bt) {
        const int kb = k0 + bt * 32;
        const int p = p_next, y = y_next;
        const unsigned cw = cw_next;
        if (bt + 1 < b1) {
            y_next = __ldg(perm + kb + 32 + lane);
            cw_next = __ldg(cwp + kb + 32 + lane);
            p_next = bpat[kb / 32 + 1];
        }
        if (p != cur) {
            flush();
            cur = p;
        }
        if (y >= 0) {
            const float self = __ldg(b + y);
            // src[u]: the mass of N_u(y) that can move into y (free, not the goal)
            float src[9];
#pragma unroll
            for (int u = 0; u < 9; ++u) {
                src[u] = 0.0f;
                if (u != 4 && !((cw >> u) & 1u)) {
                    const int x = y + step9(m, u);
                    src[u] = x == m.goal ? 0.0f : __ldg(b + x);
                }
            }
            float q[LEAF ? kA9 : 1];
            if constexpr (LEAF) {
#pragma unroll
                for (int j = 0; j < kA9; ++j) q[j] = __ldg(Q + static_cast<size_t>(j) * m.n + y);
            }
            const bool goal = y == m.goal;
#pragma unroll
            for (int a = 0; a < kA9; ++a) {
                float v;
                if (a == 4) {
                    v = self;
                } else {
                    int s1, s2;
                    slips9(a, s1, s2);
                    v = fmaf(w0, src[8 - a], w1 * (src[8 - s1] + src[8 - s2]));
                    if (goal) v += self;
                    else {
                        const float stay = w0 * static_cast<float>((cw >> a) & 1u) +
                                           w1 * static_cast<float>(((cw >> s1) & 1u) + ((cw >> s2) & 1u));
                        v = fmaf(stay, self, v);
                    }
                }
                accM[a] += v;
                accR[a] = fmaf(self, __ldg(Rt + static_cast<size_t>(a) * m.n + y), accR[a]);
                if constexpr (LEAF) {
#pragma unroll
                    for (int j = 0; j < kA9; ++j) accH[a * kA9 + j] = fmaf(v, q[j], accH[a * kA9 + j]);
                }
            }
        }
    }
    flush();
#pragma unroll
    for (int a = 0; a < kA9; ++a) {
        const float r = warp_sum(accR[a]);
        if (lane == 0) bins[w][a][kRec9 - 1] = r;
    }
    __syncthreads();
    float *out = rec + (static_cast<size_t>(i) * nchunk + c) * kA9 * kRec9;
    for (int t = threadIdx.x; t < kA9 * kRec9; t += blockDim.x) {
        const int a = t / kRec9, v = t - a * kRec9;
        if (!LEAF && v >= kZ9 && v < kRec9 - 1) continue;
        float s = 0.0f;
        for (int u = 0; u < kW9; ++u) s += bins[u][a][v];
        out[t] = s;
    }
}

// One warp per (node i, action a): the chunk records added in order,
// P(z) = sum_p O(p, z) M[p] for every z, K draws of z by the FP32 inverse
// CDF of the (level, code * 9 + a) uniform stream, the unique z in ascending
// order with their counts and P(z), and at the deepest level each unique
// z's leaf value max_a' sum_p O(p, z) H[p][a'] / P(z).
template <bool LEAF>
__global__ void __launch_bounds__(kT9) k9_finalise(M9 m, int l, int nl, int nchunk, int K, const float *__restrict__ rec,
                                                  const unsigned long long *__restrict__ code, uint64_t seed,
                                                  uint32_t episode, float *__restrict__ Rq, int *__restrict__ un,
                                                  int *__restrict__ uz, int *__restrict__ uf, float *__restrict__ upz,
                                                  float *__restrict__ uval, unsigned long long *bcount) {
    __shared__ float s_tot[kW9][kRec9];
    __shared__ float s_P[kW9][kZ9];
    __shared__ int s_z[kW9][QV9_MAX_K], s_f[kW9][QV9_MAX_K], s_n[kW9];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = blockIdx.x * kW9 + w;
    if (g >= nl * kA9) return;
    const int i = g / kA9, a = g - i * kA9;
    // record of (node i, chunk c): [9][kRec9], action a's part at a * kRec9
    const float *r = rec + static_cast<size_t>(i) * nchunk * kA9 * kRec9 + static_cast<size_t>(a) * kRec9;
    for (int v = lane; v < kRec9; v += 32) {
        if (!LEAF && v >= kZ9 && v < kRec9 - 1) continue;
        float s = 0.0f;
        for (int c = 0; c < nchunk; ++c) s += r[static_cast<size_t>(c) * kA9 * kRec9 + v];
        s_tot[w][v] = s;
    }
    __syncwarp();
    if (lane < kZ9) {
        float s = 0.0f;
        for (int p = 0; p < kZ9; ++p) s = fmaf(olik9(m.ps, p, lane), s_tot[w][p], s);
        s_P[w][lane] = s;
    }
    __syncwarp();
    if (lane == 0) {
        float C[kZ9];
        float acc = 0.0f;
        for (int z = 0; z < kZ9; ++z) {
            acc += s_P[w][z];
            C[z] = acc;
        }
        int cnt[kZ9];
        for (int z = 0; z < kZ9; ++z) cnt[z] = 0;
        const uint64_t path = code[i] * kA9 + static_cast<uint64_t>(a);
        unsigned long long nbd = 0ull;
        for (int k = 0; k < K; ++k) {
            const float u = sample_uniform(seed, episode, l, path, k);
            const float t = u * C[kZ9 - 1];
            int pick = kZ9 - 1;
            for (int z = 0; z < kZ9; ++z)
                if (t < C[z]) {
                    pick = z;
                    break;
                }
            ++cnt[pick];
            for (int z = 0; z + 1 < kZ9; ++z)
                if (fabsf(u - C[z] / C[kZ9 - 1]) < kBoundaryEps) {
                    ++nbd;
                    break;
                }
        }
        int n = 0;
        for (int z = 0; z < kZ9; ++z)
            if (cnt[z]) {
                s_z[w][n] = z;
                s_f[w][n] = cnt[z];
                ++n;
            }
        s_n[w] = n;
        Rq[g] = s_tot[w][kRec9 - 1];
        un[g] = n;
        for (int q = 0; q < n; ++q) {
            uz[static_cast<size_t>(g) * K + q] = s_z[w][q];
            uf[static_cast<size_t>(g) * K + q] = s_f[w][q];
            upz[static_cast<size_t>(g) * K + q] = s_P[w][s_z[w][q]];
        }
        if (nbd) atomicAdd(bcount, nbd);
    }
    __syncwarp();
    if constexpr (LEAF) {
        const int n = s_n[w];
        for (int q = 0; q < n; ++q) {
            const int z = s_z[w][q];
            float v = -INFINITY;
            if (lane < kA9) {
                float s = 0.0f;
                for (int p = 0; p < kZ9; ++p) s = fmaf(olik9(m.ps, p, z), s_tot[w][kZ9 + p * kA9 + lane], s);
                v = s;
            }
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) uval[static_cast<size_t>(g) * K + q] = v / s_P[w][z];
        }
    }
}

// Exclusive scan of the children counts of every (node, action) of a
// level, in (node, action) order, and the next level's size.  One CTA.
__global__ void __launch_bounds__(1024) k9_scan(int N, const int *__restrict__ un, int *__restrict__ coff,
                                               int *__restrict__ total) {
    __shared__ int s[1024];
    const int t = threadIdx.x, per = (N + 1023) / 1024;
    const int lo = min(N, t * per), hi = min(N, lo + per);
    int sum = 0;
    for (int j = lo; j < hi; ++j) sum += un[j];
    s[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = t >= o ? s[t - o] : 0;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    int run = s[t] - sum;
    for (int j = lo; j < hi; ++j) {
        coff[j] = run;
        run += un[j];
    }
    if (t == 1023) *total = s[1023];
}

// One thread per (node, action): its children's records in the next level.
__global__ void __launch_bounds__(kT9) k9_emit(int nl, int K, const int *__restrict__ un, const int *__restrict__ coff,
                                              const int *__restrict__ uz, const int *__restrict__ uf,
                                              const float *__restrict__ upz, const float *__restrict__ uval,
                                              const unsigned long long *__restrict__ code, Lvl9 next) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nl * kA9) return;
    const int i = g / kA9, a = g - i * kA9, n = un[g], c0 = coff[g];
    for (int q = 0; q < n; ++q) {
        const int j = c0 + q;
        const int z = uz[static_cast<size_t>(g) * K + q];
        next.parent[j] = i;
        next.action[j] = a;
        next.obs[j] = z;
        next.weight[j] = static_cast<float>(uf[static_cast<size_t>(g) * K + q]) / static_cast<float>(K);
        next.pz[j] = upz[static_cast<size_t>(g) * K + q];
        next.value[j] = uval ? uval[static_cast<size_t>(g) * K + q] : 0.0f;
        next.code[j] = (code[i] * kA9 + static_cast<unsigned long long>(a)) * kZ9 + static_cast<unsigned long long>(z);
    }
}

// Grid (bands, children): child j's belief, Eq. 3, b'(y) = O(p(y), z) bbar(y)
// / P(z) with bbar from the parent's belief.
__global__ void __launch_bounds__(kT9) k9_children(M9 m, const float *__restrict__ bel, Lvl9 next,
                                                  float *__restrict__ out) {
    const int j = blockIdx.y;
    const int i = next.parent[j], a = next.action[j], z = next.obs[j];
    const float inv = 1.0f / next.pz[j];
    const float *b = bel + static_cast<size_t>(i) * m.n;
    float *o = out + static_cast<size_t>(j) * m.n;
    const int y0 = blockIdx.x * kBand9, y1 = min(m.n, y0 + kBand9);
    for (int y = y0 + threadIdx.x; y < y1; y += blockDim.x) {
        const unsigned cw = m.cw[y];
        const float v = predict9(m, b, y, cw, a);
        o[y] = occ9(cw) ? 0.0f : olik9(m.ps, pattern9(cw), z) * v * inv;
    }
}

// Alg. 6 / 7 for one level: U_Q(b, a) = R(b, a) + gamma sum_children w U_V,
// U_V(b) = max_a U_Q.  One thread per node.
__global__ void __launch_bounds__(kT9) k9_backup(int nl, float gamma, const float *__restrict__ Rq,
                                                const int *__restrict__ un, const int *__restrict__ coff,
                                                const float *__restrict__ wn, const float *__restrict__ vn,
                                                float *__restrict__ UQ, float *__restrict__ value) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    float best = 0.0f;
    for (int a = 0; a < kA9; ++a) {
        const int g = i * kA9 + a, c0 = coff[g];
        float s = 0.0f;
        for (int q = 0; q < un[g]; ++q) s = fmaf(wn[c0 + q], vn[c0 + q], s);
        const float u = fmaf(gamma, s, Rq[g]);
        UQ[g] = u;
        best = (a == 0 || u > best) ? u : best;
    }
    value[i] = best;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

M9 m9_of(const qv9_model_t &md, const uint16_t *cw) {
    M9 m;
    m.H = md.H;
    m.W = md.W;
    m.n = md.H * md.W;
    m.goal = md.goal;
    m.eps = md.slip;
    m.ps = md.p_sensor;
    m.gamma = md.discount;
    m.cw = cw;
    return m;
}

}  // namespace
}  // namespace qv

struct qv9 {
    qv9_model_t model;
    int depth, K, n, Kp, nchunk_leaf, nchunk_inner;  // expansion chunks of kChunk9 / kChunkSmall9 positions
    std::vector<uint16_t> cw;
    std::vector<int> perm;
    std::vector<signed char> bpat;
    long cap[QV9_MAX_DEPTH + 1];
    long node_off[QV9_MAX_DEPTH + 2];  // node arrays: level l at node_off[l]
    long total_nodes, internal_nodes;  // all levels; levels 0 .. depth - 1
    std::vector<uint16_t> cwp;         // cell words in pattern order (0 at padding)
    size_t off_cw, off_perm, off_cwp, off_bpat, off_Rt, off_V0, off_V1, off_res, off_flags, off_bel;
    size_t off_parent, off_action, off_obs, off_weight, off_pz, off_value, off_code;
    size_t off_R, off_UQ, off_un, off_coff, off_uz, off_uf, off_upz, off_uval, off_rec;
    size_t ws_bytes;
    char *ws;
    int n_level[QV9_MAX_DEPTH + 1];
    bool planned;
};

namespace {

qv::Lvl9 level9(const qv9 *h, int l) {
    qv::Lvl9 L;
    const long o = h->node_off[l];
    L.parent = reinterpret_cast<int *>(h->ws + h->off_parent) + o;
    L.action = reinterpret_cast<int *>(h->ws + h->off_action) + o;
    L.obs = reinterpret_cast<int *>(h->ws + h->off_obs) + o;
    L.weight = reinterpret_cast<float *>(h->ws + h->off_weight) + o;
    L.pz = reinterpret_cast<float *>(h->ws + h->off_pz) + o;
    L.value = reinterpret_cast<float *>(h->ws + h->off_value) + o;
    L.code = reinterpret_cast<unsigned long long *>(h->ws + h->off_code) + o;
    return L;
}

float *belief9(const qv9 *h, int l) {
    return reinterpret_cast<float *>(h->ws + h->off_bel) + static_cast<size_t>(h->node_off[l]) * h->n;
}

}  // namespace

extern "C" qv_status qv9_create(const qv9_model_t *m, int32_t depth, int32_t K, qv9_t **out) {
    QV_RANGE("qv9_create");
    if (!m || !m->d_occ || !out) return qv_set_error(QV_ERR_INVALID, "qv9_create: null pointer");
    *out = nullptr;
    if (m->H < 1 || m->W < 1 || m->W > QV_MAX_WIDTH || m->goal < 0 || m->goal >= m->H * m->W)
        return qv_set_error(QV_ERR_INVALID, "qv9_create: bad grid");
    if (!(m->slip >= 0.0f && m->slip <= 1.0f / 3.0f) || !(m->p_sensor >= 0.5f && m->p_sensor <= 1.0f) ||
        !(m->discount > 0.0f && m->discount < 1.0f))
        return qv_set_error(QV_ERR_INVALID, "qv9_create: bad model parameters");
    if (depth < 1 || depth > QV9_MAX_DEPTH || K < 1 || K > QV9_MAX_K)
        return qv_set_error(QV_ERR_INVALID, "qv9_create: depth %d or K %d out of range", depth, K);
    const int H = m->H, W = m->W, n = H * W;
    std::vector<uint8_t> occ(n);
    if (qv_check_cuda(cudaMemcpy(occ.data(), m->d_occ, n, cudaMemcpyDeviceToHost), "occupancy") != QV_OK)
        return QV_ERR_CUDA;
    if (occ[m->goal]) return qv_set_error(QV_ERR_INVALID, "qv9_create: the goal is occupied");
    qv9 *h = new qv9();
    h->model = *m;
    h->depth = depth;
    h->K = K;
    h->n = n;
    h->cw.assign(n, 0);
    auto blocked = [&](int r, int c) { return r < 0 || r >= H || c < 0 || c >= W || occ[r * W + c]; };
    std::vector<int> pat(n, 0);
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            unsigned w = 0;
            for (int t = 0; t < 9; ++t)
                if (t != 4 && blocked(r + t / 3 - 1, c + t % 3 - 1)) w |= 1u << t;
            if (occ[r * W + c]) w |= 1u << 4;
            if (r * W + c == m->goal) w |= 1u << 9;
            h->cw[r * W + c] = static_cast<uint16_t>(w);
            pat[r * W + c] = ((w >> 1) & 1) | (((w >> 3) & 1) << 1) | (((w >> 5) & 1) << 2) | (((w >> 7) & 1) << 3);
        }
    // free cells in sensor-pattern order, grid order within a pattern, each
    // pattern's run padded to a whole warp batch
    for (int p = 0; p < QV9_NUM_OBS; ++p) {
        const size_t start = h->perm.size();
        for (int y = 0; y < n; ++y)
            if (!occ[y] && pat[y] == p) h->perm.push_back(y);
        while ((h->perm.size() - start) % qv::kRun9) h->perm.push_back(-1);
        for (size_t k = start; k < h->perm.size(); k += qv::kRun9) h->bpat.push_back(static_cast<signed char>(p));
    }
    if (h->perm.empty()) {
        h->perm.assign(qv::kRun9, -1);
        h->bpat.assign(1, 0);
    }
    h->Kp = static_cast<int>(h->perm.size());
    h->cwp.assign(h->Kp, 0);
    for (int k = 0; k < h->Kp; ++k)
        if (h->perm[k] >= 0) h->cwp[k] = h->cw[h->perm[k]];
    h->nchunk_leaf = (h->Kp + qv::kChunk9 - 1) / qv::kChunk9;
    h->nchunk_inner = (h->Kp + qv::kChunkSmall9 - 1) / qv::kChunkSmall9;
    h->cap[0] = 1;
    for (int l = 1; l <= depth; ++l) h->cap[l] = h->cap[l - 1] * qv::kA9 * std::min(K, QV9_NUM_OBS);
    h->node_off[0] = 0;
    for (int l = 0; l <= depth; ++l) h->node_off[l + 1] = h->node_off[l] + h->cap[l];
    h->total_nodes = h->node_off[depth + 1];
    h->internal_nodes = h->node_off[depth];
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = qv::a256(off + bytes);
        return o;
    };
    const size_t NT = h->total_nodes, NI = h->internal_nodes;
    h->off_cw = take(n * sizeof(uint16_t));
    h->off_perm = take(h->Kp * sizeof(int));
    h->off_cwp = take(h->Kp * sizeof(uint16_t));
    h->off_bpat = take(h->bpat.size());
    h->off_Rt = take(static_cast<size_t>(qv::kA9) * n * sizeof(float));
    h->off_V0 = take(n * sizeof(double));
    h->off_V1 = take(n * sizeof(double));
    h->off_res = take(qv::kVIResCap * sizeof(unsigned long long));
    h->off_flags = take(64);
    h->off_bel = take(NI * n * sizeof(float));
    h->off_parent = take(NT * sizeof(int));
    h->off_action = take(NT * sizeof(int));
    h->off_obs = take(NT * sizeof(int));
    h->off_weight = take(NT * sizeof(float));
    h->off_pz = take(NT * sizeof(float));
    h->off_value = take(NT * sizeof(float));
    h->off_code = take(NT * sizeof(unsigned long long));
    h->off_R = take(NI * qv::kA9 * sizeof(float));
    h->off_UQ = take(NI * qv::kA9 * sizeof(float));
    h->off_un = take(NI * qv::kA9 * sizeof(int));
    h->off_coff = take(NI * qv::kA9 * sizeof(int));
    h->off_uz = take(NI * qv::kA9 * K * sizeof(int));
    h->off_uf = take(NI * qv::kA9 * K * sizeof(int));
    h->off_upz = take(NI * qv::kA9 * K * sizeof(float));
    h->off_uval = take(NI * qv::kA9 * K * sizeof(float));
    const size_t rec_nodes = std::max(static_cast<size_t>(h->cap[depth - 1]) * h->nchunk_leaf,
                                      depth > 1 ? static_cast<size_t>(h->cap[depth - 2]) * h->nchunk_inner : 0);
    h->off_rec = take(rec_nodes * qv::kA9 * qv::kRec9 * sizeof(float));
    h->ws_bytes = off;
    h->ws = nullptr;
    h->planned = false;
    *out = h;
    return QV_OK;
}

extern "C" size_t qv9_workspace_bytes(const qv9_t *h) { return h ? h->ws_bytes : 0; }

extern "C" void qv9_destroy(qv9_t *h) { delete h; }

extern "C" qv_status qv9_set_workspace(qv9_t *h, void *d_ws, size_t ws_bytes, qv_stream_t stream) {
    if (!h || !d_ws) return qv_set_error(QV_ERR_INVALID, "qv9_set_workspace: null pointer");
    if (reinterpret_cast<uintptr_t>(d_ws) & 255)
        return qv_set_error(QV_ERR_INVALID, "qv9_set_workspace: workspace must be 256-byte aligned");
    if (ws_bytes < h->ws_bytes)
        return qv_set_error(QV_ERR_WORKSPACE, "qv9_set_workspace: %zu < %zu bytes", ws_bytes, h->ws_bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    h->ws = static_cast<char *>(d_ws);
    h->planned = false;
    if (qv_check_cuda(cudaMemcpyAsync(h->ws + h->off_cw, h->cw.data(), h->cw.size() * sizeof(uint16_t),
                                      cudaMemcpyHostToDevice, st), "cell words") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(h->ws + h->off_perm, h->perm.data(), h->perm.size() * sizeof(int),
                                      cudaMemcpyHostToDevice, st), "pattern order") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(h->ws + h->off_cwp, h->cwp.data(), h->cwp.size() * sizeof(uint16_t),
                                      cudaMemcpyHostToDevice, st), "pattern-order cell words") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(h->ws + h->off_bpat, h->bpat.data(), h->bpat.size(),
                                      cudaMemcpyHostToDevice, st), "batch patterns") != QV_OK)
        return QV_ERR_CUDA;
    const qv::M9 m = qv::m9_of(h->model, reinterpret_cast<const uint16_t *>(h->ws + h->off_cw));
    const int grid = std::max(1, std::min((h->n + qv::kT9 - 1) / qv::kT9, 4 * qv_num_sms()));
    qv::k9_reward_table<<<grid, qv::kT9, 0, st>>>(m, reinterpret_cast<float *>(h->ws + h->off_Rt));
    if (qv_check_cuda(cudaGetLastError(), "qv9 reward table") != QV_OK) return QV_ERR_CUDA;
    // the tables are read from pageable host memory: finish before returning
    return qv_check_cuda(cudaStreamSynchronize(st), "qv9_set_workspace");
}

namespace {

template <typename T>
qv_status vi9(qv9 *h, double tol, int max_sweeps, int truncated, T *d_V, float *d_Q, int *sweeps_out,
              double *residual_out, cudaStream_t st) {
    const qv::M9 m = qv::m9_of(h->model, reinterpret_cast<const uint16_t *>(h->ws + h->off_cw));
    T *V[2] = {reinterpret_cast<T *>(h->ws + h->off_V0), reinterpret_cast<T *>(h->ws + h->off_V1)};
    auto *res = reinterpret_cast<unsigned long long *>(h->ws + h->off_res);
    int *flags = reinterpret_cast<int *>(h->ws + h->off_flags);  // done, sweeps
    const int limit = truncated > 0 ? truncated : max_sweeps;
    const double t = truncated > 0 ? -1.0 : tol;
    if (qv_check_cuda(cudaMemsetAsync(V[0], 0, h->n * sizeof(T), st), "memset") != QV_OK ||
        qv_check_cuda(cudaMemsetAsync(res, 0, static_cast<size_t>(limit + 1) * sizeof(unsigned long long), st),
                      "memset") != QV_OK ||
        qv_check_cuda(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st), "memset") != QV_OK)
        return QV_ERR_CUDA;
    const int grid = std::max(1, std::min((h->n + qv::kT9 - 1) / qv::kT9, 4 * qv_num_sms()));
    int done = 0, k = 0;
    while (k < limit && !done) {
        const int k1 = std::min(limit, k + 16);
        for (; k < k1; ++k)
            qv::k9_vi_sweep<T><<<grid, qv::kT9, 0, st>>>(m, V[k & 1], V[(k + 1) & 1], k, t, res, flags, flags + 1);
        if (qv_check_cuda(cudaGetLastError(), "qv9 sweep") != QV_OK) return QV_ERR_CUDA;
        if (qv_check_cuda(cudaMemcpyAsync(&done, flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flag") != QV_OK ||
            qv_check_cuda(cudaStreamSynchronize(st), "qv9_value_iterate") != QV_OK)
            return QV_ERR_CUDA;
    }
    int n_sw = k;
    if (done && (qv_check_cuda(cudaMemcpyAsync(&n_sw, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st),
                               "sweeps") != QV_OK ||
                 qv_check_cuda(cudaStreamSynchronize(st), "qv9_value_iterate") != QV_OK))
        return QV_ERR_CUDA;
    unsigned long long rb = 0ull;
    if (n_sw > 0 && (qv_check_cuda(cudaMemcpyAsync(&rb, res + n_sw - 1, sizeof(rb), cudaMemcpyDeviceToHost, st),
                                   "residual") != QV_OK ||
                     qv_check_cuda(cudaStreamSynchronize(st), "qv9_value_iterate") != QV_OK))
        return QV_ERR_CUDA;
    double r;
    std::memcpy(&r, &rb, sizeof(r));
    qv::k9_vi_q<T><<<grid, qv::kT9, 0, st>>>(m, V[n_sw & 1], d_V, d_Q);
    if (qv_check_cuda(cudaGetLastError(), "qv9 Q") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "qv9_value_iterate") != QV_OK)
        return QV_ERR_CUDA;
    if (sweeps_out) *sweeps_out = n_sw;
    if (residual_out) *residual_out = r;
    if (truncated <= 0 && !(r < tol))
        return qv_set_error(QV_ERR_NOT_CONVERGED, "qv9_value_iterate: %d sweeps, residual %g", n_sw, r);
    return QV_OK;
}

}  // namespace

extern "C" qv_status qv9_value_iterate(qv9_t *h, int32_t dtype, double tol, int32_t max_sweeps, int32_t truncated,
                                       void *d_V, float *d_Q, int32_t *sweeps_out, double *residual_out,
                                       qv_stream_t stream) {
    QV_RANGE("qv9_value_iterate");
    if (!h || !d_V || !d_Q) return qv_set_error(QV_ERR_INVALID, "qv9_value_iterate: null pointer");
    if (!h->ws) return qv_set_error(QV_ERR_INVALID, "qv9_value_iterate: no workspace (qv9_set_workspace)");
    if (dtype != QV_F32 && dtype != QV_F64) return qv_set_error(QV_ERR_INVALID, "qv9_value_iterate: dtype");
    const int limit = truncated > 0 ? truncated : max_sweeps;
    if (limit < 1 || limit >= qv::kVIResCap)
        return qv_set_error(QV_ERR_INVALID, "qv9_value_iterate: %d sweeps outside 1..%d", limit, qv::kVIResCap - 1);
    h->planned = false;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return dtype == QV_F64 ? vi9<double>(h, tol, max_sweeps, truncated, static_cast<double *>(d_V), d_Q, sweeps_out,
                                         residual_out, st)
                           : vi9<float>(h, tol, max_sweeps, truncated, static_cast<float *>(d_V), d_Q, sweeps_out,
                                        residual_out, st);
}

extern "C" qv_status qv9_plan(qv9_t *h, const float *d_Q, const float *d_b0, uint64_t seed, uint32_t episode,
                              qv9_plan_result_t *res, qv_stream_t stream) {
    QV_RANGE("qv9_plan");
    if (!h || !d_Q || !d_b0 || !res) return qv_set_error(QV_ERR_INVALID, "qv9_plan: null pointer");
    if (!h->ws) return qv_set_error(QV_ERR_INVALID, "qv9_plan: no workspace (qv9_set_workspace)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *ws = h->ws;
    const qv::M9 m = qv::m9_of(h->model, reinterpret_cast<const uint16_t *>(ws + h->off_cw));
    const int *perm = reinterpret_cast<const int *>(ws + h->off_perm);
    const auto *cwp = reinterpret_cast<const uint16_t *>(ws + h->off_cwp);
    const float *Rt = reinterpret_cast<const float *>(ws + h->off_Rt);
    const auto *bpat = reinterpret_cast<const signed char *>(ws + h->off_bpat);
    auto *flags = reinterpret_cast<int *>(ws + h->off_flags);
    auto *bcount = reinterpret_cast<unsigned long long *>(ws + h->off_flags + 16);
    float *Rq = reinterpret_cast<float *>(ws + h->off_R);
    float *UQ = reinterpret_cast<float *>(ws + h->off_UQ);
    int *un = reinterpret_cast<int *>(ws + h->off_un);
    int *coff = reinterpret_cast<int *>(ws + h->off_coff);
    int *uz = reinterpret_cast<int *>(ws + h->off_uz);
    int *uf = reinterpret_cast<int *>(ws + h->off_uf);
    float *upz = reinterpret_cast<float *>(ws + h->off_upz);
    float *uval = reinterpret_cast<float *>(ws + h->off_uval);
    float *rec = reinterpret_cast<float *>(ws + h->off_rec);
    const int D = h->depth, K = h->K;
    h->planned = false;
    const int rgrid = std::max(1, std::min((h->n + qv::kT9 - 1) / qv::kT9, 4 * qv_num_sms()));
    qv::k9_root<<<rgrid, qv::kT9, 0, st>>>(m, d_b0, belief9(h, 0), level9(h, 0), bcount);
    h->n_level[0] = 1;
    for (int l = 0; l < D; ++l) {
        QV_RANGE("qv9_plan", l);
        const int nl = h->n_level[l];
        const bool leaf = l + 1 == D;
        const size_t q0 = static_cast<size_t>(h->node_off[l]) * qv::kA9;  // Q-node base of the level
        const int nchunk = leaf ? h->nchunk_leaf : h->nchunk_inner;
        const int clen = leaf ? qv::kChunk9 : qv::kChunkSmall9;
        const dim3 eg(nchunk, nl);
        if (leaf)
            qv::k9_expand<true><<<eg, qv::kT9, 0, st>>>(m, belief9(h, l), perm, cwp, bpat, h->Kp, clen, nchunk, d_Q,
                                                         Rt, rec);
        else
            qv::k9_expand<false><<<eg, qv::kT9, 0, st>>>(m, belief9(h, l), perm, cwp, bpat, h->Kp, clen, nchunk, d_Q,
                                                          Rt, rec);
        const int fg = (nl * qv::kA9 + qv::kW9 - 1) / qv::kW9;
        const qv::Lvl9 L = level9(h, l);
        if (leaf)
            qv::k9_finalise<true><<<fg, qv::kT9, 0, st>>>(m, l, nl, nchunk, K, rec, L.code, seed, episode, Rq + q0,
                                                          un + q0, uz + q0 * K, uf + q0 * K, upz + q0 * K,
                                                          uval + q0 * K, bcount);
        else
            qv::k9_finalise<false><<<fg, qv::kT9, 0, st>>>(m, l, nl, nchunk, K, rec, L.code, seed, episode, Rq + q0,
                                                           un + q0, uz + q0 * K, uf + q0 * K, upz + q0 * K,
                                                           uval + q0 * K, bcount);
        qv::k9_scan<<<1, 1024, 0, st>>>(nl * qv::kA9, un + q0, coff + q0, flags + 2);
        int nn = 0;
        if (qv_check_cuda(cudaGetLastError(), "qv9_plan launch") != QV_OK ||
            qv_check_cuda(cudaMemcpyAsync(&nn, flags + 2, sizeof(int), cudaMemcpyDeviceToHost, st), "count") != QV_OK ||
            qv_check_cuda(cudaStreamSynchronize(st), "qv9_plan") != QV_OK)
            return QV_ERR_CUDA;
        if (nn > h->cap[l + 1]) return qv_set_error(QV_ERR_CAPACITY, "qv9_plan: level %d holds %d > %ld", l + 1, nn,
                                                    h->cap[l + 1]);
        h->n_level[l + 1] = nn;
        const qv::Lvl9 N = level9(h, l + 1);
        qv::k9_emit<<<(nl * qv::kA9 + qv::kT9 - 1) / qv::kT9, qv::kT9, 0, st>>>(
            nl, K, un + q0, coff + q0, uz + q0 * K, uf + q0 * K, upz + q0 * K, leaf ? uval + q0 * K : nullptr, L.code,
            N);
        if (!leaf && nn > 0)
            qv::k9_children<<<dim3((h->n + qv::kBand9 - 1) / qv::kBand9, nn), qv::kT9, 0, st>>>(m, belief9(h, l), N,
                                                                                              belief9(h, l + 1));
    }
    for (int l = D - 1; l >= 0; --l) {
        QV_RANGE("qv9_plan backup", l);
        const size_t q0 = static_cast<size_t>(h->node_off[l]) * qv::kA9;
        const qv::Lvl9 L = level9(h, l), N = level9(h, l + 1);
        qv::k9_backup<<<(h->n_level[l] + qv::kT9 - 1) / qv::kT9, qv::kT9, 0, st>>>(
            h->n_level[l], h->model.discount, Rq + q0, un + q0, coff + q0, N.weight, N.value, UQ + q0, L.value);
    }
    float q[qv::kA9], v = 0.0f;
    unsigned long long nb = 0ull;
    if (qv_check_cuda(cudaGetLastError(), "qv9_plan backup") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(q, UQ, sizeof(q), cudaMemcpyDeviceToHost, st), "root") != QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&v, level9(h, 0).value, sizeof(float), cudaMemcpyDeviceToHost, st), "root") !=
            QV_OK ||
        qv_check_cuda(cudaMemcpyAsync(&nb, bcount, sizeof(nb), cudaMemcpyDeviceToHost, st), "boundary") != QV_OK ||
        qv_check_cuda(cudaStreamSynchronize(st), "qv9_plan") != QV_OK)
        return QV_ERR_CUDA;
    int best = 0;
    for (int a = 1; a < qv::kA9; ++a)
        if (q[a] > q[best]) best = a;
    res->action = best;
    res->value = v;
    for (int a = 0; a < qv::kA9; ++a) res->q[a] = q[a];
    for (int l = 0; l <= QV9_MAX_DEPTH; ++l) res->nodes_per_level[l] = l <= D ? h->n_level[l] : 0;
    res->boundary_samples = static_cast<int64_t>(nb);
    h->planned = true;
    return QV_OK;
}

extern "C" qv_status qv9_level(const qv9_t *h, int32_t level, qv9_level_view_t *out) {
    if (!h || !out) return qv_set_error(QV_ERR_INVALID, "qv9_level: null pointer");
    if (!h->planned) return qv_set_error(QV_ERR_INVALID, "qv9_level: no plan on this handle");
    if (level < 0 || level > h->depth) return qv_set_error(QV_ERR_INVALID, "qv9_level: level %d", level);
    const qv::Lvl9 L = level9(h, level);
    out->count = h->n_level[level];
    out->parent = L.parent;
    out->action = L.action;
    out->obs = L.obs;
    out->weight = L.weight;
    out->pz = L.pz;
    out->value = L.value;
    const bool internal = level < h->depth;
    out->belief = internal ? belief9(h, level) : nullptr;
    const size_t q0 = static_cast<size_t>(h->node_off[level]) * qv::kA9;
    out->R = internal ? reinterpret_cast<const float *>(h->ws + h->off_R) + q0 : nullptr;
    out->UQ = internal ? reinterpret_cast<const float *>(h->ws + h->off_UQ) + q0 : nullptr;
    return QV_OK;
}
