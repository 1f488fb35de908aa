// index.cu -- counting-sort cell index (grid environment, paper Sec. 4.1):
// cell histogram (integer atomics), single-pass exclusive scan with
// decoupled look-back, and scatter of agent ids into cell order.
#include <algorithm>

#include "amb_internal.cuh"

namespace amb {

// ------------------------------------------------------------------ scan ---
constexpr int kScanNT = 256;
constexpr int kScanRounds = 4;
constexpr uint32_t kScanTile = kScanNT * 4 * kScanRounds;  // 4096 items

__global__ void __launch_bounds__(kScanNT) scan_kernel(const int32_t *__restrict__ in, int32_t *__restrict__ out,
                                                       int32_t *__restrict__ out2, uint32_t m, uint32_t n_tiles,
                                                       unsigned long long *tickets, uint32_t parity,
                                                       uint64_t *status, uint32_t epoch, uint32_t *err)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp[kScanNT / 32 + 1];
    __shared__ uint32_t s_prefix;
    if (blockIdx.x == 0 && threadIdx.x == 0) tickets[parity ^ 1u] = 0ull;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (uint32_t)atomicAdd(&tickets[parity], 1ull);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if (tile >= n_tiles) break;
        const uint64_t base = (uint64_t)tile * kScanTile;
        uint32_t v[kScanRounds][4];
        uint32_t excl[kScanRounds];
        uint32_t running = 0;
#pragma unroll
        for (int r = 0; r < kScanRounds; ++r) {
            const uint64_t i0 = base + ((uint64_t)r * kScanNT + threadIdx.x) * 4u;
            if (i0 + 3 < m) {
                const int4 q = *reinterpret_cast<const int4 *>(in + i0);
                v[r][0] = (uint32_t)q.x; v[r][1] = (uint32_t)q.y; v[r][2] = (uint32_t)q.z; v[r][3] = (uint32_t)q.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) v[r][e] = (i0 + e < m) ? (uint32_t)in[i0 + e] : 0u;
            }
            const uint32_t tsum = v[r][0] + v[r][1] + v[r][2] + v[r][3];
            uint32_t total;
            const uint32_t ex = block_exclusive_scan<kScanNT>(tsum, s_warp, &total);
            excl[r] = running + ex;
            running += total;
        }
        if (threadIdx.x == 0) s_prefix = lookback_exclusive(status, tile, epoch, running, err);
        __syncthreads();
        const uint32_t pre = s_prefix;
#pragma unroll
        for (int r = 0; r < kScanRounds; ++r) {
            const uint64_t i0 = base + ((uint64_t)r * kScanNT + threadIdx.x) * 4u;
            uint32_t e0 = pre + excl[r];
            uint32_t o[4];
            o[0] = e0; o[1] = o[0] + v[r][0]; o[2] = o[1] + v[r][1]; o[3] = o[2] + v[r][2];
            if (i0 + 3 < m) {
                const int4 q = make_int4((int)o[0], (int)o[1], (int)o[2], (int)o[3]);
                *reinterpret_cast<int4 *>(out + i0) = q;
                if (out2) *reinterpret_cast<int4 *>(out2 + i0) = q;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < m) {
                        out[i0 + e] = (int32_t)o[e];
                        if (out2) out2[i0 + e] = (int32_t)o[e];
                    }
            }
        }
        if (tile == n_tiles - 1 && threadIdx.x == 0) out[m] = (int32_t)(pre + running);
    }
}

amb_status Lookback::ensure(size_t tiles, cudaStream_t s)
{
    if (!tickets) {
        AMB_TRY(dalloc(&tickets, 2, s));
        AMB_TRY_CUDA(cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned long long), s));
    }
    if (tiles > cap) {
        size_t c = cap ? cap : 1024;
        while (c < tiles) c *= 2;
        if (status) dfree(status, s);
        AMB_TRY(dalloc(&status, c, s));
        // zero epoch == "not ready" for every epoch in use
        AMB_TRY_CUDA(cudaMemsetAsync(status, 0, c * sizeof(uint64_t), s));
        cap = c;
    }
    return AMB_OK;
}

void Lookback::release(cudaStream_t s)
{
    dfree(status, s);
    dfree(tickets, s);
    cap = 0;
}

amb_status launch_scan(const int32_t *in, int32_t *out, int32_t *out2, uint32_t m, Lookback &lb, uint32_t *err,
                       cudaStream_t s)
{
    const uint32_t n_tiles = (uint32_t)(((uint64_t)m + kScanTile - 1) / kScanTile);
    if (n_tiles == 0) {
        AMB_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return AMB_OK;
    }
    AMB_TRY(lb.ensure(n_tiles, s));
    uint32_t parity, epoch;
    lb.next(&parity, &epoch);
    const unsigned sms = device_sms();
    const unsigned grid = (unsigned)std::min<uint64_t>(n_tiles, (uint64_t)sms * 8u);
    scan_kernel<<<grid, kScanNT, 0, s>>>(in, out, out2, m, n_tiles, lb.tickets, parity, lb.status, epoch, err);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

uint32_t scan_tiles(uint32_t m) { return (uint32_t)(((uint64_t)m + kScanTile - 1) / kScanTile); }

// ------------------------------------------------------ histogram/scatter ---
__global__ void cell_hist_kernel(const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n,
                                 int32_t L, int32_t *__restrict__ cnt, uint32_t *err)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t xi = x[i], yi = y[i];
        if ((uint32_t)xi >= (uint32_t)L || (uint32_t)yi >= (uint32_t)L) {
            atomicOr(err, ERR_RANGE);
            continue;
        }
        atomicAdd(&cnt[(uint32_t)yi * (uint32_t)L + (uint32_t)xi], 1);
    }
}

__global__ void cell_scatter_kernel(const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n,
                                    int32_t L, int32_t *__restrict__ cursor, int32_t *__restrict__ ids)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t xi = x[i], yi = y[i];
        if ((uint32_t)xi >= (uint32_t)L || (uint32_t)yi >= (uint32_t)L) continue;
        const int32_t pos = atomicAdd(&cursor[(uint32_t)yi * (uint32_t)L + (uint32_t)xi], 1);
        ids[pos] = (int32_t)i;
    }
}

amb_status launch_cell_scatter(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *cursor,
                               int32_t *ids, cudaStream_t s)
{
    if (n == 0) return AMB_OK;
    cell_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, (int32_t)L, cursor, ids);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_cell_index_raw(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *start,
                                 int32_t *ids, int32_t *cnt, int32_t *cursor, uint64_t *status,
                                 unsigned long long *tickets, uint32_t parity, uint32_t epoch, uint32_t *err,
                                 cudaStream_t s)
{
    const uint64_t C = (uint64_t)L * L;
    const uint32_t n_tiles = scan_tiles((uint32_t)C);
    AMB_TRY_CUDA(cudaMemsetAsync(cnt, 0, C * sizeof(int32_t), s));
    if (n) {
        cell_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, (int32_t)L, cnt, err);
        AMB_TRY_CUDA(cudaGetLastError());
    }
    const unsigned sms = device_sms();
    const unsigned grid = (unsigned)std::min<uint64_t>(n_tiles, (uint64_t)sms * 8u);
    scan_kernel<<<grid, kScanNT, 0, s>>>(cnt, start, cursor, (uint32_t)C, n_tiles, tickets, parity, status, epoch, err);
    AMB_TRY_CUDA(cudaGetLastError());
    if (n) {
        cell_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, (int32_t)L, cursor, ids);
        AMB_TRY_CUDA(cudaGetLastError());
    }
    return AMB_OK;
}

amb_status launch_cell_index(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *start,
                             int32_t *ids, int32_t *cnt, int32_t *cursor, Lookback &lb, uint32_t *err,
                             cudaStream_t s)
{
    const uint64_t C = (uint64_t)L * L;
    AMB_TRY_CUDA(cudaMemsetAsync(cnt, 0, C * sizeof(int32_t), s));
    if (n) {
        cell_hist_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, (int32_t)L, cnt, err);
        AMB_TRY_CUDA(cudaGetLastError());
    }
    AMB_TRY(launch_scan(cnt, start, cursor, (uint32_t)C, lb, err, s));
    if (n) {
        cell_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, y, n, (int32_t)L, cursor, ids);
        AMB_TRY_CUDA(cudaGetLastError());
    }
    return AMB_OK;
}

}  // namespace amb
