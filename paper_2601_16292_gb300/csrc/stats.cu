// stats.cu -- end-of-run statistics and invariant checks (paper Sec. 5.1.3 /
// 6.2 invariants; summary statistics as exact integer sums followed by one
// double division each).
#include "amb_internal.cuh"

namespace amb {

// min, max and sum of an int32 column: out = {min, max} (int32), sum (int64)
__global__ void minmax_sum_kernel(const int32_t *__restrict__ v, uint32_t n, int32_t *__restrict__ mm,
                                  unsigned long long *__restrict__ sum)
{
    int32_t lo = INT32_MAX, hi = INT32_MIN;
    long long s = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t a = v[i];
        lo = min(lo, a);
        hi = max(hi, a);
        s += a;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_down_sync(0xffffffffu, hi, o));
        s += __shfl_down_sync(0xffffffffu, s, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
        atomicAdd(sum, (unsigned long long)s);
    }
}

__global__ void value_hist_kernel(const int32_t *__restrict__ v, uint32_t n, int32_t base, uint32_t bins,
                                  unsigned long long *__restrict__ hist)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t b = (uint32_t)((int64_t)v[i] - base);
        if (b < bins) atomicAdd(&hist[b], 1ull);
    }
}

// Gini numerator from the value histogram (ascending values base + b):
// agents of bin b hold ranks a+1 .. a+h (a = agents in lower bins), and
// sum over those ranks of (2i - n - 1) = h (2a + h - n).  One block.
constexpr int kGiniNT = 1024;
__global__ void __launch_bounds__(kGiniNT) gini_numerator_kernel(const unsigned long long *__restrict__ hist,
                                                                 uint32_t bins, int32_t base, uint32_t n,
                                                                 long long *__restrict__ out /* hi, lo */)
{
    __shared__ uint32_t s_warp[kGiniNT / 32 + 1];
    __shared__ unsigned long long s_lo[kGiniNT / 32];
    __shared__ long long s_hi[kGiniNT / 32];
    __int128 acc = 0;
    uint32_t before = 0;  // agents in bins of earlier chunks
    for (uint32_t c0 = 0; c0 < bins; c0 += kGiniNT) {
        const uint32_t b = c0 + threadIdx.x;
        const uint32_t h = (b < bins) ? (uint32_t)hist[b] : 0u;
        uint32_t chunk_total;
        const uint32_t ex = block_exclusive_scan<kGiniNT>(h, s_warp, &chunk_total);
        if (h) {
            const int64_t a = (int64_t)before + ex;
            const __int128 f = (__int128)h * (__int128)(2 * a + (int64_t)h - (int64_t)n);
            acc += f * (__int128)((int64_t)base + (int64_t)b);
        }
        before += chunk_total;
    }
    // block reduction of the 128-bit partial sums as (hi, lo) pairs
    unsigned long long lo = (unsigned long long)acc;
    long long hi = (long long)(acc >> 64);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, o);
        const long long ohi = __shfl_down_sync(0xffffffffu, hi, o);
        const unsigned long long nlo = lo + olo;
        hi = hi + ohi + (nlo < lo ? 1 : 0);
        lo = nlo;
    }
    if (lane == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long L = 0;
        long long H = 0;
        for (int q = 0; q < kGiniNT / 32; ++q) {
            const unsigned long long nl = L + s_lo[q];
            H = H + s_hi[q] + (nl < L ? 1 : 0);
            L = nl;
        }
        out[0] = H;
        out[1] = (long long)L;
    }
}

// Occupancy per cell from id-ordered positions.
__global__ void occupancy_kernel(const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n, int32_t L,
                                 int32_t *__restrict__ occ)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t xi = x[i], yi = y[i];
        if ((uint32_t)xi < (uint32_t)L && (uint32_t)yi < (uint32_t)L)
            atomicAdd(&occ[(uint32_t)yi * (uint32_t)L + (uint32_t)xi], 1);
    }
}

// Occupancy per cell from the index: occ[c] = start[c+1] - start[c].
__global__ void occupancy_from_start_kernel(const int32_t *__restrict__ start, uint64_t C, int32_t *__restrict__ occ)
{
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < C; c += (uint64_t)gridDim.x * blockDim.x)
        occ[c] = start[c + 1] - start[c];
}

// Histogram of an int32 array of nonnegative values (bins = max + 1).
__global__ void count_hist_kernel(const int32_t *__restrict__ v, uint64_t m, uint32_t bins,
                                  unsigned long long *__restrict__ hist)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = (uint32_t)v[i];
        if (b < bins) atomicAdd(&hist[b], 1ull);
    }
}

__global__ void max_kernel(const int32_t *__restrict__ v, uint64_t m, int32_t *__restrict__ out)
{
    int32_t hi = INT32_MIN;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
        hi = max(hi, v[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hi = max(hi, __shfl_down_sync(0xffffffffu, hi, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, hi);
}

// Curve sums over the per-step series (column I = 1): S0, S1, S2 as 128-bit
// (hi, lo) pairs, the peak and the first step reaching it.  One block.
constexpr int kCurveNT = 256;
__global__ void __launch_bounds__(kCurveNT) curve_sums_kernel(const int64_t *__restrict__ series, uint32_t T,
                                                              long long *__restrict__ out /* 8 */)
{
    __shared__ unsigned long long s_lo[3][kCurveNT];
    __shared__ unsigned long long s_hi[3][kCurveNT];
    __shared__ long long s_pk[kCurveNT];
    __shared__ uint32_t s_am[kCurveNT];
    unsigned __int128 a0 = 0, a1 = 0, a2 = 0;
    long long pk = -1;
    uint32_t am = 0;
    for (uint32_t j = threadIdx.x; j < T; j += kCurveNT) {
        const unsigned long long v = (unsigned long long)series[(size_t)j * 4u + 1u];
        const unsigned long long t = (unsigned long long)j + 1ull;
        a0 += v;
        a1 += (unsigned __int128)v * t;
        a2 += (unsigned __int128)v * t * t;
        if ((long long)v > pk) {
            pk = (long long)v;
            am = (uint32_t)t;
        }
    }
    s_lo[0][threadIdx.x] = (unsigned long long)a0; s_hi[0][threadIdx.x] = (unsigned long long)(a0 >> 64);
    s_lo[1][threadIdx.x] = (unsigned long long)a1; s_hi[1][threadIdx.x] = (unsigned long long)(a1 >> 64);
    s_lo[2][threadIdx.x] = (unsigned long long)a2; s_hi[2][threadIdx.x] = (unsigned long long)(a2 >> 64);
    s_pk[threadIdx.x] = pk;
    s_am[threadIdx.x] = am;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned __int128 r[3] = {0, 0, 0};
        long long P = -1;
        uint32_t A = 0;
        for (int q = 0; q < kCurveNT; ++q) {
            for (int j = 0; j < 3; ++j) r[j] += ((unsigned __int128)s_hi[j][q] << 64) | s_lo[j][q];
            // earliest step among equal peaks
            if (s_pk[q] > P || (s_pk[q] == P && s_am[q] < A && s_pk[q] >= 0)) {
                P = s_pk[q];
                A = s_am[q];
            }
        }
        for (int j = 0; j < 3; ++j) {
            out[2 * j] = (long long)(unsigned long long)(r[j] >> 64);
            out[2 * j + 1] = (long long)(unsigned long long)r[j];
        }
        out[6] = P;
        out[7] = (long long)A;
    }
}

// Checks: coordinates in range (walk/SIR id-ordered), index monotone.
__global__ void bounds_check_kernel(const int32_t *__restrict__ x, const int32_t *__restrict__ y, uint32_t n,
                                    int32_t L, unsigned long long *__restrict__ bad)
{
    uint32_t b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b += ((uint32_t)x[i] >= (uint32_t)L || (uint32_t)y[i] >= (uint32_t)L);
    if (b) atomicAdd(bad, (unsigned long long)b);
}

__global__ void monotone_check_kernel(const int32_t *__restrict__ start, uint64_t C, unsigned long long *__restrict__ bad)
{
    uint32_t b = 0;
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < C; c += (uint64_t)gridDim.x * blockDim.x)
        b += (start[c + 1] < start[c]);
    if (b) atomicAdd(bad, (unsigned long long)b);
}

__global__ void state_count_kernel(const uint8_t *__restrict__ st, uint32_t n, unsigned long long *__restrict__ cnt /* 4 */)
{
    uint32_t c[4] = {0, 0, 0, 0};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t s = st[i];
        c[s < 3 ? s : 3] += 1;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t v = c[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&cnt[j], (unsigned long long)v);
    }
}

// ------------------------------------------------------------ host side ---
amb_status launch_minmax_sum(const int32_t *v, uint32_t n, int32_t *mm, unsigned long long *sum, cudaStream_t s)
{
    const int32_t init[2] = {INT32_MAX, INT32_MIN};
    AMB_TRY_CUDA(cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s));
    AMB_TRY_CUDA(cudaMemsetAsync(sum, 0, sizeof(unsigned long long), s));
    if (n) minmax_sum_kernel<<<grid_for(n, 256, 8u), 256, 0, s>>>(v, n, mm, sum);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_value_hist(const int32_t *v, uint32_t n, int32_t base, uint32_t bins, unsigned long long *hist,
                             cudaStream_t s)
{
    AMB_TRY_CUDA(cudaMemsetAsync(hist, 0, (size_t)bins * sizeof(unsigned long long), s));
    if (n) value_hist_kernel<<<grid_for(n, 256, 8u), 256, 0, s>>>(v, n, base, bins, hist);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_gini_numerator(const unsigned long long *hist, uint32_t bins, int32_t base, uint32_t n,
                                 long long *out, cudaStream_t s)
{
    gini_numerator_kernel<<<1, kGiniNT, 0, s>>>(hist, bins, base, n, out);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_occupancy(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *occ, cudaStream_t s)
{
    const uint64_t C = (uint64_t)L * L;
    AMB_TRY_CUDA(cudaMemsetAsync(occ, 0, C * sizeof(int32_t), s));
    if (n) occupancy_kernel<<<grid_for(n, 256, 8u), 256, 0, s>>>(x, y, n, (int32_t)L, occ);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_occupancy_from_start(const int32_t *start, uint64_t C, int32_t *occ, cudaStream_t s)
{
    occupancy_from_start_kernel<<<grid_for(C, 256, 8u), 256, 0, s>>>(start, C, occ);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_max(const int32_t *v, uint64_t m, int32_t *out, cudaStream_t s)
{
    const int32_t init = INT32_MIN;
    AMB_TRY_CUDA(cudaMemcpyAsync(out, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    if (m) max_kernel<<<grid_for(m, 256, 8u), 256, 0, s>>>(v, m, out);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_count_hist(const int32_t *v, uint64_t m, uint32_t bins, unsigned long long *hist, cudaStream_t s)
{
    AMB_TRY_CUDA(cudaMemsetAsync(hist, 0, (size_t)bins * sizeof(unsigned long long), s));
    if (m) count_hist_kernel<<<grid_for(m, 256, 8u), 256, 0, s>>>(v, m, bins, hist);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_curve_sums(const int64_t *series, uint32_t T, long long *out, cudaStream_t s)
{
    curve_sums_kernel<<<1, kCurveNT, 0, s>>>(series, T, out);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_bounds_check(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, unsigned long long *bad,
                               cudaStream_t s)
{
    if (n) bounds_check_kernel<<<grid_for(n, 256, 8u), 256, 0, s>>>(x, y, n, (int32_t)L, bad);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_monotone_check(const int32_t *start, uint64_t C, unsigned long long *bad, cudaStream_t s)
{
    if (C) monotone_check_kernel<<<grid_for(C, 256, 8u), 256, 0, s>>>(start, C, bad);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_state_count(const uint8_t *st, uint32_t n, unsigned long long *cnt, cudaStream_t s)
{
    AMB_TRY_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s));
    if (n) state_count_kernel<<<grid_for(n, 256, 8u), 256, 0, s>>>(st, n, cnt);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

}  // namespace amb
