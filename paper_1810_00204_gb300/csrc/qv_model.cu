// qv_model.cu -- model build (Sec. II): per-cell words encoding the blocked-move
// rule of Eq. 10, the inflow pattern of the motion stencil, the beacon label
// and the free flag.
#include "qv_common.cuh"

namespace qv {

__global__ void __launch_bounds__(256)
k_model_build(int H, int W, int P, const uint8_t *__restrict__ occ, const int32_t *__restrict__ beacons,
              int B, int sense_range, int goal, uint16_t *__restrict__ cell) {
    __shared__ int s_br[QV_MAX_BEACONS], s_bc[QV_MAX_BEACONS];
    for (int k = threadIdx.x; k < B; k += blockDim.x) {
        s_br[k] = beacons[k] / P;
        s_bc[k] = beacons[k] % P;
    }
    __syncthreads();
    const int n = H * P;
    for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < n; y += gridDim.x * blockDim.x) {
        const int r = y / P, c = y - r * P;
        auto is_free = [&](int rr, int cc) {
            return rr >= 0 && rr < H && cc >= 0 && cc < W && occ[rr * P + cc] == 0;
        };
        const bool f = is_free(r, c);
        const int dr[4] = {-1, 0, 1, 0}, dc[4] = {0, 1, 0, -1};
        unsigned blocked = 0, inflow = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            const int rr = r + dr[d], cc = c + dc[d];
            const bool nf = is_free(rr, cc);
            if (!nf) blocked |= 1u << d;
            if (f && nf && (rr * P + cc) != goal) inflow |= 1u << d;
        }
        // nearest beacon within range, ties to the lower id, else null = B
        int best = B, bestd = 1 << 30;
        for (int k = 0; k < B; ++k) {
            const int d = abs(s_br[k] - r) + abs(s_bc[k] - c);
            if (d <= sense_range && d < bestd) {
                best = k;
                bestd = d;
            }
        }
        cell[y] = static_cast<uint16_t>(blocked | (inflow << 4) | (static_cast<unsigned>(best) << 8) |
                                        ((f ? 1u : 0u) << 15));
    }
}

}  // namespace qv

extern "C" qv_status qv_model_build(int32_t H, int32_t W, int32_t pitch, const uint8_t *d_occ,
                                    const int32_t *d_beacons, int32_t B, int32_t sense_range,
                                    int32_t goal, uint16_t *d_cell, qv_stream_t stream) {
    QV_RANGE("qv_model_build");
    if (H < 1 || W < 1 || W > QV_MAX_WIDTH || pitch != QV_PITCH(W))
        return qv_set_error(QV_ERR_INVALID, "qv_model_build: bad grid %dx%d pitch %d", H, W, pitch);
    if (B < 1 || B > QV_MAX_BEACONS)
        return qv_set_error(QV_ERR_INVALID, "qv_model_build: B=%d outside 1..%d", B, QV_MAX_BEACONS);
    if (!d_occ || !d_beacons || !d_cell)
        return qv_set_error(QV_ERR_INVALID, "qv_model_build: null pointer");
    if (goal < 0 || goal >= H * pitch || goal % pitch >= W)
        return qv_set_error(QV_ERR_INVALID, "qv_model_build: goal %d outside the grid", goal);
    if (sense_range < 0) return qv_set_error(QV_ERR_INVALID, "qv_model_build: negative range");
    const long long n = static_cast<long long>(H) * pitch;
    const int grid = static_cast<int>(std::min<long long>((n + 255) / 256, 8 * qv_num_sms()));
    qv::k_model_build<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(H, W, pitch, d_occ, d_beacons, B,
                                                                          sense_range, goal, d_cell);
    return qv_check_cuda(cudaGetLastError(), "qv_model_build launch");
}
