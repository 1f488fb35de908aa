// models.cu -- per-step kernels of the three models over id-ordered columns:
//  * random walk: a full-population map (paper Listing 1 pattern), k steps
//    fused in registers (agents are independent);
//  * wealth transfer (paper Listings 2-3): filtered debit of the donors
//    (wealth > 0 on the snapshot) compacted with warp ballot / popc, and an
//    id-indexed scatter-add credit with integer atomics; one CTA keeps the
//    whole column in shared memory for all k steps when it fits, otherwise
//    two grid-wide kernels per step;
//  * SIR, generic path: move + cell histogram, counting-sort index, and the
//    infection / recovery pass reading the per-cell infected counts.
#include <algorithm>

#include "amb_internal.cuh"

namespace amb {

// --------------------------------------------------------------- walk ------
__global__ void __launch_bounds__(256) walk_kernel(int32_t *__restrict__ x, int32_t *__restrict__ y, uint32_t n,
                                                   int32_t L, uint32_t k0, uint32_t k1, uint32_t t0, uint32_t k,
                                                   uint32_t *err, int64_t *__restrict__ rows)
{
    // per-step rows {n, 0, 0, 0}: the agent count never changes
    if (blockIdx.x == 0)
        for (uint32_t j = threadIdx.x; j < k; j += blockDim.x) {
            rows[(size_t)j * 4u] = n;
            rows[(size_t)j * 4u + 1] = 0;
            rows[(size_t)j * 4u + 2] = 0;
            rows[(size_t)j * 4u + 3] = 0;
        }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
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

amb_status walk_steps(amb_pop *pop, uint32_t k)
{
    const uint32_t n = pop->p.n;
    if (k == 0) return AMB_OK;
    walk_kernel<<<grid_for(n, 256, 32u), 256, 0, pop->stream>>>(
        pop->x, pop->y, n, (int32_t)pop->p.grid_side, pop->key0, pop->key1, (uint32_t)pop->t, k, pop->err,
        pop->series + (size_t)pop->t * 4u);
    AMB_TRY_CUDA(cudaGetLastError());
    pop->launches += 1;
    return AMB_OK;
}

// ------------------------------------------------------------- wealth ------
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

__global__ void __launch_bounds__(kWealthNT) wealth_smem_kernel(int32_t *__restrict__ wg, uint32_t n, uint32_t k0,
                                                                uint32_t k1, uint32_t t0, uint32_t k,
                                                                int64_t *__restrict__ series)
{
    wealth_cta_steps(wg, n, k0, k1, t0, k, series);
}

// ------------------------------------------------------- wealth batches ---
// Device descriptor of one wealth population in a batch.
struct WealthJob {
    int32_t *w;
    int32_t *credit;  // large populations
    int64_t *series;  // row 0 = the population's step 0
    uint32_t n, k0, k1, t, t_end, pad;
};

// Small populations: one CTA per job runs all its remaining steps.
__global__ void __launch_bounds__(kWealthNT) wealth_batch_small_kernel(WealthJob *__restrict__ jobs,
                                                                       const uint32_t *__restrict__ list)
{
    WealthJob &j = jobs[list[blockIdx.x]];
    if (j.t < j.t_end) wealth_cta_steps(j.w, j.n, j.k0, j.k1, j.t, j.t_end - j.t, j.series + (size_t)j.t * 4u);
}

constexpr uint32_t kWealthChunk = 2048;  // agents per block in the batched grid-wide kernels

__device__ __forceinline__ uint32_t chunk_job(const uint32_t *prefix, uint32_t n_jobs, uint32_t g)
{
    uint32_t lo = 0, hi = n_jobs - 1;  // last job whose first chunk <= g
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Large populations, one step: donors credit their recipients (phase 1).
__global__ void __launch_bounds__(256) wealth_batch_donate_kernel(const WealthJob *__restrict__ jobs,
                                                                  const uint32_t *__restrict__ list,
                                                                  const uint32_t *__restrict__ prefix, uint32_t n_jobs)
{
    __shared__ uint32_t s_job;
    if (threadIdx.x == 0) s_job = chunk_job(prefix, n_jobs, blockIdx.x);
    __syncthreads();
    const WealthJob &j = jobs[list[s_job]];
    if (j.t >= j.t_end) return;
    const uint32_t first = (blockIdx.x - prefix[s_job]) * kWealthChunk;
    const uint32_t last = min(first + kWealthChunk, j.n);
    uint32_t local = 0;
    for (uint32_t i = first + threadIdx.x; i < last; i += blockDim.x) {
        if (j.w[i] > 0) {
            const U4 u = philox(i, j.t, j.k0, j.k1);
            uint32_t r = below(u.w0, j.n - 1u);
            r += (r >= i) ? 1u : 0u;
            atomicAdd(&j.credit[r], 1);
            ++local;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local)
        atomicAdd(reinterpret_cast<unsigned long long *>(&j.series[(size_t)j.t * 4u]), (unsigned long long)local);
}

// Large populations, one step: w' = w - [w > 0] + credit (phase 2).
__global__ void __launch_bounds__(256) wealth_batch_apply_kernel(const WealthJob *__restrict__ jobs,
                                                                 const uint32_t *__restrict__ list,
                                                                 const uint32_t *__restrict__ prefix, uint32_t n_jobs)
{
    __shared__ uint32_t s_job;
    if (threadIdx.x == 0) s_job = chunk_job(prefix, n_jobs, blockIdx.x);
    __syncthreads();
    const WealthJob &j = jobs[list[s_job]];
    if (j.t >= j.t_end) return;
    const uint32_t first = (blockIdx.x - prefix[s_job]) * kWealthChunk;
    const uint32_t last = min(first + kWealthChunk, j.n);
    long long part = 0;
    for (uint32_t i = first + threadIdx.x; i < last; i += blockDim.x) {
        const int32_t wi = j.w[i];
        const int32_t nw = (int32_t)((uint32_t)wi - (wi > 0 ? 1u : 0u) + (uint32_t)j.credit[i]);
        j.w[i] = nw;
        j.credit[i] = 0;
        part += nw;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part)
        atomicAdd(reinterpret_cast<unsigned long long *>(&j.series[(size_t)j.t * 4u + 1u]), (unsigned long long)part);
}

__global__ void wealth_batch_advance_kernel(WealthJob *__restrict__ jobs, const uint32_t *__restrict__ list,
                                            uint32_t n_jobs)
{
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_jobs; q += gridDim.x * blockDim.x) {
        WealthJob &j = jobs[list[q]];
        if (j.t < j.t_end) j.t += 1u;
    }
}

// Host side: a set of wealth populations advanced together.
amb_status wealth_batch_build(WealthBatch &wb, amb_pop **pops, const uint32_t *steps, uint32_t n, cudaStream_t s)
{
    std::vector<WealthJob> jobs(n);
    std::vector<uint32_t> small, large, prefix(1, 0u);
    size_t smem = 16;
    for (uint32_t q = 0; q < n; ++q) {
        amb_pop *p = pops[q];
        WealthJob &j = jobs[q];
        j.w = p->w;
        j.credit = p->credit;
        j.series = p->series;
        j.n = p->p.n;
        j.k0 = p->key0;
        j.k1 = p->key1;
        j.t = (uint32_t)p->t;
        j.t_end = (uint32_t)(p->t + steps[q]);
        j.pad = 0;
        if (p->p.n == 0 || steps[q] == 0) continue;
        if (wealth_uses_smem(p->p.n)) {
            small.push_back(q);
            smem = std::max(smem, (size_t)((p->p.n + 7u) & ~7u) * 4u + (size_t)p->p.n * 2u + 16u);
        } else {
            large.push_back(q);
            prefix.push_back(prefix.back() + (p->p.n + kWealthChunk - 1u) / kWealthChunk);
        }
    }
    wb.n_jobs = n;
    wb.n_small = (uint32_t)small.size();
    wb.n_large = (uint32_t)large.size();
    wb.large_chunks = prefix.back();
    wb.smem = smem;
    AMB_TRY(dalloc(reinterpret_cast<unsigned char **>(&wb.d_jobs), (size_t)n * sizeof(WealthJob), s));
    AMB_TRY(dalloc(&wb.d_small, small.size(), s));
    AMB_TRY(dalloc(&wb.d_large, large.size(), s));
    AMB_TRY(dalloc(&wb.d_prefix, prefix.size(), s));
    AMB_TRY_CUDA(cudaMemcpyAsync(wb.d_jobs, jobs.data(), (size_t)n * sizeof(WealthJob), cudaMemcpyHostToDevice, s));
    if (!small.empty())
        AMB_TRY_CUDA(cudaMemcpyAsync(wb.d_small, small.data(), small.size() * 4u, cudaMemcpyHostToDevice, s));
    if (!large.empty())
        AMB_TRY_CUDA(cudaMemcpyAsync(wb.d_large, large.data(), large.size() * 4u, cudaMemcpyHostToDevice, s));
    AMB_TRY_CUDA(cudaMemcpyAsync(wb.d_prefix, prefix.data(), prefix.size() * 4u, cudaMemcpyHostToDevice, s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
    return AMB_OK;
}

// Every small job, all of its steps (one launch).
amb_status wealth_batch_small(WealthBatch &wb, cudaStream_t s, uint64_t *launches)
{
    if (wb.n_small == 0) return AMB_OK;
    AMB_TRY_CUDA(cudaFuncSetAttribute(wealth_batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)wb.smem));
    wealth_batch_small_kernel<<<wb.n_small, kWealthNT, wb.smem, s>>>(static_cast<WealthJob *>(wb.d_jobs), wb.d_small);
    AMB_TRY_CUDA(cudaGetLastError());
    *launches += 1;
    return AMB_OK;
}

// One step of every large job (three launches).
amb_status wealth_batch_large_step(WealthBatch &wb, cudaStream_t s, uint64_t *launches)
{
    if (wb.n_large == 0) return AMB_OK;
    WealthJob *jobs = static_cast<WealthJob *>(wb.d_jobs);
    wealth_batch_donate_kernel<<<wb.large_chunks, 256, 0, s>>>(jobs, wb.d_large, wb.d_prefix, wb.n_large);
    wealth_batch_apply_kernel<<<wb.large_chunks, 256, 0, s>>>(jobs, wb.d_large, wb.d_prefix, wb.n_large);
    wealth_batch_advance_kernel<<<grid_for(wb.n_large, 128), 128, 0, s>>>(jobs, wb.d_large, wb.n_large);
    AMB_TRY_CUDA(cudaGetLastError());
    *launches += 3;
    return AMB_OK;
}

void wealth_batch_release(WealthBatch &wb, cudaStream_t s)
{
    void *j = wb.d_jobs;
    dfree(j, s);
    wb.d_jobs = nullptr;
    dfree(wb.d_small, s);
    dfree(wb.d_large, s);
    dfree(wb.d_prefix, s);
}

// Grid-wide path, phase 1: donors on the snapshot credit their recipient.
__global__ void __launch_bounds__(256) wealth_donate_kernel(const int32_t *__restrict__ w, int32_t *__restrict__ credit,
                                                            uint32_t n, uint32_t k0, uint32_t k1, uint32_t t,
                                                            int64_t *__restrict__ row)
{
    uint32_t local = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (w[i] > 0) {
            const U4 u = philox(i, t, k0, k1);
            uint32_t r = below(u.w0, n - 1u);
            r += (r >= i) ? 1u : 0u;
            atomicAdd(&credit[r], 1);
            ++local;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(reinterpret_cast<unsigned long long *>(&row[0]), (unsigned long long)local);
}

// Grid-wide path, phase 2: w' = w - [w > 0] + credit; credit cleared.
__global__ void __launch_bounds__(256) wealth_apply_kernel(int32_t *__restrict__ w, int32_t *__restrict__ credit,
                                                           uint32_t n, int64_t *__restrict__ row)
{
    long long part = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t wi = w[i];
        const int32_t nw = (int32_t)((uint32_t)wi - (wi > 0 ? 1u : 0u) + (uint32_t)credit[i]);
        w[i] = nw;
        credit[i] = 0;
        part += nw;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) atomicAdd(reinterpret_cast<unsigned long long *>(&row[1]), (unsigned long long)part);
}

__global__ void wealth_total_kernel(const int32_t *__restrict__ w, uint32_t n, int64_t *__restrict__ row)
{
    long long part = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) part += w[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0 && part) atomicAdd(reinterpret_cast<unsigned long long *>(&row[1]), (unsigned long long)part);
}

bool wealth_uses_smem(uint32_t n) { return n <= kWealthSmemMaxN; }

amb_status wealth_steps(amb_pop *pop, uint32_t k)
{
    const uint32_t n = pop->p.n;
    int64_t *rows = pop->series + (size_t)pop->t * 4u;
    if (k == 0) return AMB_OK;
    AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)k * 4u * sizeof(int64_t), pop->stream));
    if (n == 0) return AMB_OK;
    if (wealth_uses_smem(n)) {
        const size_t smem = (size_t)((n + 7u) & ~7u) * 4u + (size_t)n * 2u + 16u;
        AMB_TRY_CUDA(cudaFuncSetAttribute(wealth_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        wealth_smem_kernel<<<1, kWealthNT, smem, pop->stream>>>(pop->w, n, pop->key0, pop->key1, (uint32_t)pop->t, k,
                                                                rows);
        AMB_TRY_CUDA(cudaGetLastError());
        pop->launches += 1;
        return AMB_OK;
    }
    const unsigned g = grid_for(n, 256, 16u);
    for (uint32_t s = 0; s < k; ++s) {
        int64_t *row = rows + (size_t)s * 4u;
        if (n >= 2) {
            wealth_donate_kernel<<<g, 256, 0, pop->stream>>>(pop->w, pop->credit, n, pop->key0, pop->key1,
                                                             (uint32_t)(pop->t + s), row);
            wealth_apply_kernel<<<g, 256, 0, pop->stream>>>(pop->w, pop->credit, n, row);
            pop->launches += 2;
        } else {
            wealth_total_kernel<<<g, 256, 0, pop->stream>>>(pop->w, n, row);
            pop->launches += 1;
        }
        AMB_TRY_CUDA(cudaGetLastError());
    }
    return AMB_OK;
}

// ------------------------------------------------------ SIR generic path ---
// Move every agent; count agents (cnt) and start-of-step infected (inf) per
// new cell.
__global__ void __launch_bounds__(256) sir_move_count_kernel(int32_t *__restrict__ x, int32_t *__restrict__ y,
                                                             const uint8_t *__restrict__ state, uint32_t n, int32_t L,
                                                             uint32_t k0, uint32_t k1, uint32_t t,
                                                             int32_t *__restrict__ cnt, int32_t *__restrict__ inf,
                                                             uint32_t *err)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int32_t xi = x[i], yi = y[i];
        if ((uint32_t)xi >= (uint32_t)L || (uint32_t)yi >= (uint32_t)L) {
            atomicOr(err, ERR_RANGE);
            continue;
        }
        const U4 u = philox(i, t, k0, k1);
        const uint32_t d = u.w0 >> 29;
        xi = ring_add(xi, dir_dx(d), L);
        yi = ring_add(yi, dir_dy(d), L);
        x[i] = xi;
        y[i] = yi;
        const uint32_t c = (uint32_t)yi * (uint32_t)L + (uint32_t)xi;
        atomicAdd(&cnt[c], 1);
        if (state[i] == AMB_I) atomicAdd(&inf[c], 1);
    }
}

// Transitions against the start-of-step states; counts S, I, R, new
// infections into the step's row (warp-aggregated).
__global__ void __launch_bounds__(256) sir_transition_kernel(const int32_t *__restrict__ x,
                                                             const int32_t *__restrict__ y,
                                                             uint8_t *__restrict__ state, uint32_t n, int32_t L,
                                                             uint32_t k0, uint32_t k1, uint32_t t,
                                                             const int32_t *__restrict__ inf,
                                                             const uint32_t *__restrict__ t_inf, uint32_t K,
                                                             uint32_t t_rec, int64_t *__restrict__ row)
{
    uint32_t cs = 0, ci = 0, cr = 0, cn = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t s = state[i];
        const U4 u = philox(i, t, k0, k1);
        if (s == AMB_S) {
            const uint32_t k = (uint32_t)inf[(uint32_t)y[i] * (uint32_t)L + (uint32_t)x[i]];
            if (k >= 1u && u.w1 < t_inf[k < K ? k : K]) {
                s = AMB_I;
                ++cn;
            }
        } else if (s == AMB_I) {
            if (u.w2 < t_rec) s = AMB_R;
        }
        state[i] = (uint8_t)s;
        cs += (s == AMB_S);
        ci += (s == AMB_I);
        cr += (s == AMB_R);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cs += __shfl_down_sync(0xffffffffu, cs, o);
        ci += __shfl_down_sync(0xffffffffu, ci, o);
        cr += __shfl_down_sync(0xffffffffu, cr, o);
        cn += __shfl_down_sync(0xffffffffu, cn, o);
    }
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *r = reinterpret_cast<unsigned long long *>(row);
        if (cs) atomicAdd(&r[0], (unsigned long long)cs);
        if (ci) atomicAdd(&r[1], (unsigned long long)ci);
        if (cr) atomicAdd(&r[2], (unsigned long long)cr);
        if (cn) atomicAdd(&r[3], (unsigned long long)cn);
    }
}

amb_status sir_generic_steps(amb_pop *pop, uint32_t k)
{
    const uint32_t n = pop->p.n, L = pop->p.grid_side;
    const uint64_t C = (uint64_t)L * L;
    int64_t *rows = pop->series + (size_t)pop->t * 4u;
    if (k == 0) return AMB_OK;
    AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)k * 4u * sizeof(int64_t), pop->stream));
    const unsigned g = grid_for(n, 256, 16u);
    for (uint32_t s = 0; s < k; ++s) {
        const uint32_t t = (uint32_t)(pop->t + s);
        AMB_TRY_CUDA(cudaMemsetAsync(pop->cnt, 0, C * sizeof(int32_t), pop->stream));
        AMB_TRY_CUDA(cudaMemsetAsync(pop->inf, 0, C * sizeof(int32_t), pop->stream));
        if (n) {
            sir_move_count_kernel<<<g, 256, 0, pop->stream>>>(pop->x, pop->y, pop->state, n, (int32_t)L, pop->key0,
                                                              pop->key1, t, pop->cnt, pop->inf, pop->err);
            AMB_TRY_CUDA(cudaGetLastError());
            pop->launches += 1;
        }
        // counting-sort index of the new positions
        AMB_TRY(launch_scan(pop->cnt, pop->start, pop->cursor, (uint32_t)C, pop->lb, pop->err, pop->stream));
        pop->launches += 1;
        if (n) {
            AMB_TRY(launch_cell_scatter(pop->x, pop->y, n, L, pop->cursor, pop->ids, pop->stream));
            sir_transition_kernel<<<g, 256, 0, pop->stream>>>(pop->x, pop->y, pop->state, n, (int32_t)L, pop->key0,
                                                              pop->key1, t, pop->inf, pop->t_inf_d, pop->K,
                                                              pop->t_rec, rows + (size_t)s * 4u);
            AMB_TRY_CUDA(cudaGetLastError());
            pop->launches += 2;
        }
    }
    pop->index_valid = true;
    return AMB_OK;
}

}  // namespace amb
