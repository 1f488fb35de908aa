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

#include <cooperative_groups.h>

#include "wealth_device.cuh"

namespace amb {

// --------------------------------------------------------------- walk ------
__global__ void __launch_bounds__(256) walk_kernel(int32_t *__restrict__ x, int32_t *__restrict__ y, uint32_t n,
                                                   int32_t L, uint32_t k0, uint32_t k1, uint32_t t0, uint32_t k,
                                                   uint32_t *err, int64_t *__restrict__ rows)
{
    if (blockIdx.x == 0) walk_rows(rows, n, k);
    const uint32_t per = (n + gridDim.x - 1u) / gridDim.x;
    const uint32_t first = min(n, blockIdx.x * per), last = min(n, first + per);
    walk_range(x, y, first, last, L, k0, k1, t0, k, err);
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
__global__ void __launch_bounds__(kWealthNT) wealth_smem_kernel(int32_t *__restrict__ wg, uint32_t n, uint32_t k0,
                                                                uint32_t k1, uint32_t t0, uint32_t k,
                                                                int64_t *__restrict__ series)
{
    wealth_cta_steps(wg, n, k0, k1, t0, k, series);
}

// Grid-wide path, phase 1: donors on the snapshot credit their recipient.
__global__ void __launch_bounds__(256) wealth_donate_kernel(const int32_t *__restrict__ w, int32_t *__restrict__ credit,
                                                            uint32_t n, uint32_t k0, uint32_t k1, uint32_t t,
                                                            int64_t *__restrict__ row)
{
    const uint32_t per = (n + gridDim.x - 1u) / gridDim.x;
    const uint32_t first = min(n, blockIdx.x * per);
    wealth_donate_range(w, credit, n, k0, k1, t, first, min(n, first + per), row);
}

// Grid-wide path, phase 2: w' = w - [w > 0] + credit; credit cleared.
__global__ void __launch_bounds__(256) wealth_apply_kernel(int32_t *__restrict__ w, int32_t *__restrict__ credit,
                                                           uint32_t n, int64_t *__restrict__ row)
{
    const uint32_t per = (n + gridDim.x - 1u) / gridDim.x;
    const uint32_t first = min(n, blockIdx.x * per);
    wealth_apply_range(w, credit, first, min(n, first + per), row);
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

// ------------------------------------------------- wealth, one cluster ---
// All k steps of a column of n agents (kClusterMinN <= n <= kWealthSmemMaxN)
// on one thread-block cluster: CTA q of the cluster keeps agents
// [q per, (q+1) per) in its shared memory, with two credit arrays used in
// alternate steps.  Step t, every CTA, its own agents only: fold in the
// credits of step t-1, take the donors on that snapshot, debit them, and add
// one unit to each recipient's credit word of step t in the owning CTA's
// shared memory (distributed shared memory atomics); then one cluster
// barrier.  Credits of step t land in the other array than those being
// folded, and a CTA can only start step t+1 after every CTA has passed step
// t's barrier, i.e. finished folding step t-1's credits, so one barrier per
// step suffices.  The total after step t is summed while step t+1 folds (a
// final fold after the last step).
constexpr int kClusterNT = 256;
constexpr uint32_t kClusterMinN = 4096;

__global__ void __launch_bounds__(kClusterNT) wealth_cluster_kernel(int32_t *__restrict__ wg, uint32_t n, uint32_t per,
                                                                    uint32_t inv_per, uint32_t k0, uint32_t k1,
                                                                    uint32_t t0, uint32_t k, int64_t *__restrict__ rows)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) int32_t cl_smem[];
    __shared__ long long s_red[kClusterNT / 32];
    __shared__ uint32_t s_donors[kClusterNT / 32];
    int32_t *w = cl_smem;            // own agents
    int32_t *cr0 = cl_smem + per;    // credits of even steps
    int32_t *cr1 = cl_smem + 2 * per;  // credits of odd steps
    const uint32_t q = cluster.block_rank();
    const uint32_t lo = q * per, hi = min(n, lo + per), mine = hi > lo ? hi - lo : 0u;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    for (uint32_t i = tid; i < per; i += kClusterNT) {
        w[i] = i < mine ? wg[lo + i] : 0;
        cr0[i] = 0;
        cr1[i] = 0;
    }
    cluster.sync();
    for (uint32_t s = 0; s <= k; ++s) {  // s = k: the final fold
        const uint32_t t = t0 + s;
        int32_t *fold = ((t & 1u) ? cr0 : cr1);   // credits of step t-1
        int32_t *give = ((t & 1u) ? cr1 : cr0);   // credits of step t
        long long total = 0;
        uint32_t donors = 0;
        for (uint32_t i = tid; i < mine; i += kClusterNT) {
            int32_t wi = (int32_t)((uint32_t)w[i] + (uint32_t)fold[i]);
            fold[i] = 0;
            total += wi;
            if (s < k && n >= 2 && wi > 0) {
                wi -= 1;
                ++donors;
                const uint32_t id = lo + i;
                const U4 u = philox(id, t, k0, k1);
                uint32_t r = below(u.w0, n - 1u);
                r += (r >= id) ? 1u : 0u;
                const uint32_t owner = __umulhi(r, inv_per);  // r / per, exact for these sizes
                int32_t *dst = cluster.map_shared_rank(give, owner);
                atomicAdd(dst + (r - owner * per), 1);
            }
            w[i] = wi;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            total += __shfl_down_sync(0xffffffffu, total, o);
            donors += __shfl_down_sync(0xffffffffu, donors, o);
        }
        if (lane == 0) {
            s_red[warp] = total;
            s_donors[warp] = donors;
        }
        __syncthreads();
        if (tid == 0) {
            long long tt = 0;
            uint32_t dd = 0;
            for (int j = 0; j < kClusterNT / 32; ++j) {
                tt += s_red[j];
                dd += s_donors[j];
            }
            // the total after step t-1 (the folded snapshot), the donors of step t
            if (s > 0 && tt) atomicAdd(reinterpret_cast<unsigned long long *>(&rows[(size_t)(s - 1) * 4u + 1u]),
                                       (unsigned long long)tt);
            if (s < k && dd) atomicAdd(reinterpret_cast<unsigned long long *>(&rows[(size_t)s * 4u]),
                                       (unsigned long long)dd);
        }
        if (s < k) cluster.sync();
    }
    for (uint32_t i = tid; i < mine; i += kClusterNT) wg[lo + i] = w[i];
}

// One launch of wealth_cluster_kernel: 16 CTAs per cluster where the device
// allows it, else 8.
static amb_status wealth_cluster_steps(amb_pop *pop, uint32_t k, int64_t *rows)
{
    const uint32_t n = pop->p.n;
    static int cluster_size = 0;  // chosen on the first launch
    for (int c : {16, 8}) {
        if (cluster_size && c != cluster_size) continue;
        const uint32_t per = (n + (uint32_t)c - 1u) / (uint32_t)c;
        const uint32_t inv_per = (uint32_t)((0x100000000ull + per - 1u) / per);  // ceil(2^32 / per)
        const size_t smem = (size_t)per * 3u * sizeof(int32_t);
        if (cudaFuncSetAttribute(wealth_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, c > 8) !=
                cudaSuccess ||
            cudaFuncSetAttribute(wealth_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(kClusterNT);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = pop->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, wealth_cluster_kernel, &cfg) != cudaSuccess || clusters < 1) {
            (void)cudaGetLastError();
            continue;
        }
        const cudaError_t e = cudaLaunchKernelEx(&cfg, wealth_cluster_kernel, pop->w, n, per, inv_per, pop->key0,
                                                 pop->key1, (uint32_t)pop->t, k, rows);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cluster_size = c;
        return AMB_OK;
    }
    return fail(AMB_ECUDA, "no thread-block cluster configuration could be launched");
}

amb_status wealth_steps(amb_pop *pop, uint32_t k)
{
    const uint32_t n = pop->p.n;
    int64_t *rows = pop->series + (size_t)pop->t * 4u;
    if (k == 0) return AMB_OK;
    AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)k * 4u * sizeof(int64_t), pop->stream));
    if (n == 0) return AMB_OK;
    if (n >= kClusterMinN && wealth_uses_smem(n)) {
        AMB_TRY(wealth_cluster_steps(pop, k, rows));
        pop->launches += 1;
        return AMB_OK;
    }
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
