// wealth_device.cuh -- device code of the wealth-transfer step (paper
// Sec. 5.1.2, Listings 2-3) shared by the single-population kernels
// (models.cu) and the persistent batch kernel (batch.cu): the whole column in
// one CTA's shared memory for all steps, and the two phases of a step over a
// range of agents of a larger column (donors credit their recipients; then
// w' = w - [w > 0] + credit).  Columns that other CTAs of the same launch
// write are read through L2 (ld.global.cg), never through a possibly stale L1
// line.
#pragma once

#include "amb_internal.cuh"

namespace amb {

constexpr int kWealthNT = 1024;
// w (4 B) + donor list (2 B) per agent in shared memory
constexpr uint32_t kWealthSmemMaxN = 36864;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One CTA, whole column resident in shared memory, k steps.
__device__ __forceinline__ void wealth_cta_steps(int32_t *__restrict__ wg, uint32_t n, uint32_t k0, uint32_t k1,
                                                 uint32_t t0, uint32_t k, int64_t *__restrict__ series)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *w = reinterpret_cast<int32_t *>(smem_raw);
    const uint32_t n_pad = (n + 7u) & ~7u;
    uint16_t *donors = reinterpret_cast<uint16_t *>(w + n_pad);
    __shared__ uint32_t s_nd;
    __shared__ long long s_red[kWealthNT / 32];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = kWealthNT / 32;
    for (uint32_t i = threadIdx.x; i < n; i += kWealthNT) w[i] = wg[i];
    for (uint32_t s = 0; s < k; ++s) {
        const uint32_t t = t0 + s;
        if (threadIdx.x == 0) s_nd = 0;
        __syncthreads();
        uint32_t nd = 0;
        if (n >= 2) {
            // filtered view: donors = {w > 0} on the snapshot, compacted per warp;
            // each agent is read and debited only by its own lane here
            for (uint32_t base = (uint32_t)warp * 32u; base < n; base += NW * 32u) {
                const uint32_t i = base + (uint32_t)lane;
                const bool pred = (i < n) && (w[i] > 0);
                const uint32_t mask = __ballot_sync(0xffffffffu, pred);
                if (mask) {
                    uint32_t off = 0;
                    if (lane == 0) off = atomicAdd(&s_nd, (uint32_t)__popc(mask));
                    off = __shfl_sync(0xffffffffu, off, 0);
                    if (pred) {
                        donors[off + (uint32_t)__popc(mask & lanemask_lt())] = (uint16_t)i;
                        w[i] -= 1;
                    }
                }
            }
            __syncthreads();
            nd = s_nd;
            // scatter view: one unit to a uniformly chosen other agent
            for (uint32_t j = threadIdx.x; j < nd; j += kWealthNT) {
                const uint32_t i = donors[j];
                const U4 u = philox(i, t, k0, k1);
                uint32_t r = below(u.w0, n - 1u);
                r += (r >= i) ? 1u : 0u;
                atomicAdd(&w[r], 1);
            }
            __syncthreads();
        }
        // total wealth after the step
        long long part = 0;
        for (uint32_t i = threadIdx.x; i < n; i += kWealthNT) part += w[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) s_red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tot = 0;
            for (int q = 0; q < NW; ++q) tot += s_red[q];
            int64_t *row = series + (size_t)s * 4u;
            row[0] = (int64_t)nd;
            row[1] = tot;
            row[2] = 0;
            row[3] = 0;
        }
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < n; i += kWealthNT) wg[i] = w[i];
}

// Device descriptor of one wealth population in a batch.
struct WealthJob {
    int32_t *w;
    int32_t *credit;  // large populations: zero between steps
    int64_t *series;  // row 0 = the population's step 0
    uint32_t n, k0, k1, t, t_end, pad;
};

// Phase 1 of step t over agents [first, last) of a column of n agents (all
// threads of the block): every donor (w > 0 on the snapshot) gives one unit
// to r = r' + (r' >= i), r' = hi32(u0 (n - 1)); the donors are added to
// row[0].  Each thread loads its (up to) kRangeU agents of a pass together.
constexpr int kRangeU = 8;

__device__ __forceinline__ void wealth_donate_range(const int32_t *w, int32_t *credit, uint32_t n, uint32_t k0,
                                                    uint32_t k1, uint32_t t, uint32_t first, uint32_t last,
                                                    int64_t *row)
{
    uint32_t local = 0;
    for (uint32_t i0 = first + threadIdx.x; i0 < last; i0 += blockDim.x * kRangeU) {
        int32_t v[kRangeU];
#pragma unroll
        for (int u = 0; u < kRangeU; ++u) {
            const uint32_t i = i0 + (uint32_t)u * blockDim.x;
            v[u] = i < last ? __ldcg(&w[i]) : 0;
        }
#pragma unroll
        for (int u = 0; u < kRangeU; ++u) {
            const uint32_t i = i0 + (uint32_t)u * blockDim.x;
            if (v[u] > 0) {
                const U4 d = philox(i, t, k0, k1);
                uint32_t r = below(d.w0, n - 1u);
                r += (r >= i) ? 1u : 0u;
                atomicAdd(&credit[r], 1);
                ++local;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(reinterpret_cast<unsigned long long *>(&row[0]), (unsigned long long)local);
}

// Phase 2 over agents [first, last): w' = w - [w > 0] + credit, credit
// cleared; the new total is added to row[1].
__device__ __forceinline__ void wealth_apply_range(int32_t *w, int32_t *credit, uint32_t first, uint32_t last,
                                                   int64_t *row)
{
    long long part = 0;
    for (uint32_t i0 = first + threadIdx.x; i0 < last; i0 += blockDim.x * kRangeU) {
        int32_t v[kRangeU], c[kRangeU];
#pragma unroll
        for (int u = 0; u < kRangeU; ++u) {
            const uint32_t i = i0 + (uint32_t)u * blockDim.x;
            v[u] = i < last ? __ldcg(&w[i]) : 0;
            c[u] = i < last ? __ldcg(&credit[i]) : 0;
        }
#pragma unroll
        for (int u = 0; u < kRangeU; ++u) {
            const uint32_t i = i0 + (uint32_t)u * blockDim.x;
            if (i < last) {
                const int32_t nw = (int32_t)((uint32_t)v[u] - (v[u] > 0 ? 1u : 0u) + (uint32_t)c[u]);
                w[i] = nw;
                credit[i] = 0;
                part += nw;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) atomicAdd(reinterpret_cast<unsigned long long *>(&row[1]), (unsigned long long)part);
}

// k steps of the random walk (Moore moves on the torus, paper Sec. 5.1.2
// re-cast on the grid of Sec. 4.1) for agents [first, last), fused in
// registers (all threads of the block).
__device__ __forceinline__ void walk_range(int32_t *x, int32_t *y, uint32_t first, uint32_t last, int32_t L,
                                           uint32_t k0, uint32_t k1, uint32_t t0, uint32_t k, uint32_t *err)
{
    for (uint32_t i = first + threadIdx.x; i < last; i += blockDim.x) {
        int32_t xi = x[i], yi = y[i];
        if ((uint32_t)xi >= (uint32_t)L || (uint32_t)yi >= (uint32_t)L) {
            atomicOr(err, ERR_RANGE);
            continue;
        }
        for (uint32_t s = 0; s < k; ++s) {
            const U4 u = philox(i, t0 + s, k0, k1);
            const uint32_t d = u.w0 >> 29;
            xi = ring_add(xi, dir_dx(d), L);
            yi = ring_add(yi, dir_dy(d), L);
        }
        x[i] = xi;
        y[i] = yi;
    }
}

// The walk's per-step rows {n, 0, 0, 0} for steps 0 .. k-1 of `rows` (the
// agent count never changes).
__device__ __forceinline__ void walk_rows(int64_t *rows, uint32_t n, uint32_t k)
{
    for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
        rows[(size_t)j * 4u] = n;
        rows[(size_t)j * 4u + 1] = 0;
        rows[(size_t)j * 4u + 2] = 0;
        rows[(size_t)j * 4u + 3] = 0;
    }
}

}  // namespace amb
