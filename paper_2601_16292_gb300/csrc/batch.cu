// batch.cu -- many independent simulation jobs advanced together (the
// paper's Experiment / ParallelRunner, Sec. 4.2, re-cast for one GPU) by
// persistent kernel launches: one CTA per SM takes work units from a device
// queue until every job has taken all of its steps.  The SIR jobs, the small
// wealth jobs and the other jobs take one launch each, one after the other,
// because a launch takes the largest shared memory its jobs need.
//
// Queue.  An entry is a piece of work made of `units` independent units:
//   * one step of a SIR job (units = its bands, taken in band order, each
//     band's output slot found by decoupled look-back inside the step);
//   * phase 1 or phase 2 of one step of a large wealth job (units = chunks of
//     32,768 agents: donors credit their recipients; w' = w - [w > 0] + credit);
//   * all steps of a small wealth job (one unit: the column in one CTA's
//     shared memory);
//   * all steps of a walk job (units = chunks of 32,768 agents, steps fused).
// A CTA claims the next unit of the head entry with one atomic; when the
// entry's units are all claimed the head moves on.  The CTA that completes
// the last unit of an entry publishes the job's next entry at the tail (the
// next step, or phase 2 after phase 1): a job's steps follow one another,
// while the steps of different jobs overlap freely.  Every entry that will
// ever exist is counted up front, so the queue never overflows, and no unit
// waits for one that has not been claimed (the only waits are the look-back
// on earlier bands of the same step, and an idle CTA's wait for the next
// entry to be published by a unit in progress); every wait is bounded.
//
// Data that other CTAs of the launch wrote (the records and row tables of
// the previous step, job descriptors, wealth columns) are read through L2,
// never through a possibly stale L1 line.  An autotuner picks the band shape
// of the SIR jobs by timing candidates on throwaway copies of a sample of
// the jobs (results do not depend on it).
#include <algorithm>
#include <new>
#include <vector>

#include "band_device.cuh"
#include "wealth_device.cuh"

namespace amb {

enum : uint32_t { kKindSir = 0, kKindWealthSmall = 1, kKindDonate = 2, kKindApply = 3, kKindWalk = 4 };
constexpr uint32_t kUnitAgents = 32768;             // agents per unit of wealth phases and walks
constexpr uint64_t kIdleLimitNs = 4ull * kSpinLimitNs;  // an idle CTA gives up after waiting this long

struct SirJob {
    BandArgs a;           // the job's current step: buffers, step t, its count row, look-back words
    uint32_t t_end;       // the step at which the job stops
    uint32_t epoch_base;  // epoch of step t is (epoch_base + t) % 0x3FFFFFFF + 1
    uint32_t pad[2];
};

struct WalkJob {
    int32_t *x, *y;
    int64_t *rows;  // the count row of step t0
    uint32_t *err;
    uint32_t n, L, k0, k1, t0, k, pad[2];
};

struct QEntry {
    uint32_t kind, job, units, ready;
};

struct PersistArgs {
    SirJob *sir;
    WealthJob *wealth;
    WalkJob *walk;
    const uint32_t *codes;  // per SIR job: its CodeTables (kCodeWords words)
    QEntry *queue;
    uint32_t *claimed, *done;
    uint32_t *ctl;  // [0] head, [1] tail, [2] error word of the launch
    uint32_t n_entries;
    uint32_t *wide;
    uint32_t wide_words;
};

constexpr uint32_t kCodeWords = 512;
static_assert(sizeof(CodeTables) <= kCodeWords * 4u, "code tables fit their slot");

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: the next unit (entry h, unit u of e.units), or false when every
// entry has been claimed (or an idle wait ran out: the launch's error word
// gets ERR_TIMEOUT).  h_out / e_out hold the entry of the CTA's last claim on
// entry: while that entry still has units, one atomic claims the next.
__device__ bool claim_unit(const PersistArgs &pa, uint32_t &h_out, uint32_t &u_out, QEntry &e_out, bool have)
{
    if (have) {
        const uint32_t u = atomicAdd(&pa.claimed[h_out], 1u);
        if (u < e_out.units) {
            u_out = u;
            return true;
        }
    }
    uint64_t t_wait = 0;
    unsigned backoff = 32;
    for (;;) {
        const uint32_t h = ld_acquire(&pa.ctl[0]);
        if (h >= pa.n_entries) return false;
        if (ld_acquire(&pa.queue[h].ready)) {
            QEntry e;
            e.kind = __ldcg(&pa.queue[h].kind);
            e.job = __ldcg(&pa.queue[h].job);
            e.units = __ldcg(&pa.queue[h].units);
            const uint32_t u = atomicAdd(&pa.claimed[h], 1u);
            if (u < e.units) {
                h_out = h;
                u_out = u;
                e_out = e;
                return true;
            }
            atomicCAS(&pa.ctl[0], h, h + 1u);  // every unit of h is taken: move the head on
            t_wait = 0;
            continue;
        }
        // entry h is not published yet: a unit in progress will publish it
        const uint64_t now = global_ns();
        if (t_wait == 0) t_wait = now;
        if (now - t_wait > kIdleLimitNs || (error_word(&pa.ctl[2]) & ERR_TIMEOUT)) {
            atomicOr(&pa.ctl[2], ERR_TIMEOUT);
            return false;
        }
        __nanosleep(backoff);
        if (backoff < 2048) backoff <<= 1;
    }
}

// Thread 0: append the job's next entry.
__device__ __forceinline__ void publish(const PersistArgs &pa, uint32_t kind, uint32_t job, uint32_t units)
{
    const uint32_t slot = atomicAdd(&pa.ctl[1], 1u);
    if (slot >= pa.n_entries) {  // cannot happen: every entry is counted up front
        atomicOr(&pa.ctl[2], ERR_OVERFLOW);
        return;
    }
    QEntry *q = &pa.queue[slot];
    q->kind = kind;
    q->job = job;
    q->units = units;
    __threadfence();
    st_release(&q->ready, 1u);
}

// Thread 0, after the last unit of an entry: advance the job and publish
// what follows.
__device__ void entry_done(const PersistArgs &pa, const QEntry &e)
{
    if (e.kind == kKindSir) {
        SirJob *j = &pa.sir[e.job];
        BandArgs *a = &j->a;
        const uint2 *rec_in = reinterpret_cast<const uint2 *>(__ldcg(reinterpret_cast<const unsigned long long *>(&a->rec_in)));
        const int32_t *row_in = reinterpret_cast<const int32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&a->row_in)));
        uint2 *rec_out = reinterpret_cast<uint2 *>(__ldcg(reinterpret_cast<const unsigned long long *>(&a->rec_out)));
        int32_t *row_out = reinterpret_cast<int32_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&a->row_out)));
        int64_t *row = reinterpret_cast<int64_t *>(__ldcg(reinterpret_cast<const unsigned long long *>(&a->row)));
        const uint32_t t = __ldcg(&a->t) + 1u;
        a->rec_in = rec_out;
        a->row_in = row_out;
        a->rec_out = const_cast<uint2 *>(rec_in);
        a->row_out = const_cast<int32_t *>(row_in);
        a->row = row + 4;
        a->t = t;
        if (t < __ldcg(&j->t_end)) publish(pa, kKindSir, e.job, e.units);
    } else if (e.kind == kKindDonate) {
        publish(pa, kKindApply, e.job, e.units);
    } else if (e.kind == kKindApply) {
        WealthJob *w = &pa.wealth[e.job];
        const uint32_t t = __ldcg(&w->t) + 1u;
        w->t = t;
        if (t < __ldcg(&w->t_end)) publish(pa, kKindDonate, e.job, e.units);
    }
}

template <class T>
__device__ __forceinline__ void load_l2(T &dst, const T *src)
{
    static_assert(sizeof(T) % 4 == 0, "whole words");
    constexpr uint32_t kWords = sizeof(T) / 4u;
    static_assert(kWords <= kBandNT, "one word per thread");
    if (threadIdx.x < kWords)
        reinterpret_cast<uint32_t *>(&dst)[threadIdx.x] = __ldcg(reinterpret_cast<const uint32_t *>(src) + threadIdx.x);
}

__global__ void __launch_bounds__(kBandNT, 1) persist_kernel(const PersistArgs pa)
{
    extern __shared__ __align__(16) uint32_t dyn_smem[];
    __shared__ BandShared sh;
    __shared__ SirJob s_sir;
    __shared__ WealthJob s_w;
    __shared__ WalkJob s_walk;
    __shared__ QEntry s_e;
    __shared__ uint32_t s_h, s_u, s_go, s_code_job, s_desc_h;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        s_code_job = 0xFFFFFFFFu;
        s_desc_h = 0xFFFFFFFFu;  // entry whose job descriptor is in shared memory
        s_go = 0u;
    }
    if (tid < 4) sh.cnt[tid] = 0ull;
    Tally tl = {0u, 0u, 0u, 0u};
    uint32_t *wide_slice = pa.wide ? pa.wide + (size_t)blockIdx.x * pa.wide_words : nullptr;
    if (tid == 0) {
        QEntry e;
        uint32_t h = 0, u = 0;
        s_go = claim_unit(pa, h, u, e, false) ? 1u : 0u;
        s_h = h;
        s_u = u;
        s_e = e;
    }
    __syncthreads();
    for (;;) {
        if (!s_go) break;
        const QEntry e = s_e;
        const uint32_t u = s_u;
        // a job's descriptor changes only after every unit of its entry is
        // done, so it is reloaded only when the entry changes
        const bool fresh_desc = s_h != s_desc_h;
        if (e.kind == kKindSir) {
            if (fresh_desc) load_l2(s_sir, &pa.sir[e.job]);
            __syncthreads();
            if (tid == 0) {
                s_sir.a.epoch = ((s_sir.epoch_base + s_sir.a.t) % 0x3FFFFFFFu) + 1u;
                s_desc_h = s_h;
            }
            if (e.job != s_code_job) {
                const uint32_t *src = pa.codes + (size_t)e.job * kCodeWords;
                uint32_t *dst = reinterpret_cast<uint32_t *>(&sh.ct);
                for (uint32_t i = tid; i < sizeof(CodeTables) / 4u; i += kBandNT) dst[i] = src[i];
            }
            __syncthreads();
            if (tid == 0) s_code_job = e.job;
            const BandArgs &a = s_sir.a;
            process_band<false, true>(a, sh, dyn_smem, wide_slice, u, tl);
            flush_tally(sh, tl, a.row);
        } else if (e.kind == kKindWalk) {
            if (fresh_desc) load_l2(s_walk, &pa.walk[e.job]);
            __syncthreads();
            if (tid == 0) s_desc_h = s_h;
            const WalkJob &k = s_walk;
            if (u == 0) walk_rows(k.rows, k.n, k.k);
            const uint32_t first = u * kUnitAgents;
            walk_range(k.x, k.y, first, min(k.n, first + kUnitAgents), (int32_t)k.L, k.k0, k.k1, k.t0, k.k, k.err);
        } else {
            if (fresh_desc) load_l2(s_w, &pa.wealth[e.job]);
            __syncthreads();
            if (tid == 0) s_desc_h = s_h;
            const WealthJob &w = s_w;
            if (e.kind == kKindWealthSmall) {
                wealth_cta_steps(w.w, w.n, w.k0, w.k1, w.t, w.t_end - w.t, w.series + (size_t)w.t * 4u);
            } else {
                const uint32_t first = u * kUnitAgents, last = min(w.n, first + kUnitAgents);
                int64_t *row = w.series + (size_t)w.t * 4u;
                if (e.kind == kKindDonate)
                    wealth_donate_range(w.w, w.credit, w.n, w.k0, w.k1, w.t, first, last, row);
                else
                    wealth_apply_range(w.w, w.credit, first, last, row);
            }
        }
        // the unit's writes are visible GPU-wide before it is counted done;
        // the next unit of the same entry is claimed by an atomic issued
        // together with the count (a claim that has to wait for an entry to
        // be published comes only after the count, which may publish it)
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            const uint32_t u_next = atomicAdd(&pa.claimed[s_h], 1u);
            if (atomicAdd(&pa.done[s_h], 1u) + 1u == e.units) {
                __threadfence();
                entry_done(pa, e);
            }
            if (u_next < e.units) {
                s_u = u_next;
            } else {
                QEntry ne = e;
                uint32_t h = s_h, u = 0;
                s_go = claim_unit(pa, h, u, ne, false) ? 1u : 0u;
                s_h = h;
                s_u = u;
                s_e = ne;
            }
        }
        __syncthreads();
    }
}

// One block per SIR job: its code tables (load_code_tables) into global memory.
__global__ void code_tables_kernel(const uint32_t *const *__restrict__ t_inf, const uint32_t *__restrict__ K,
                                   uint32_t *__restrict__ out)
{
    __shared__ CodeTables ct;
    load_code_tables(ct, t_inf[blockIdx.x], K[blockIdx.x]);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&ct);
    uint32_t *dst = out + (size_t)blockIdx.x * kCodeWords;
    for (uint32_t i = threadIdx.x; i < sizeof(CodeTables) / 4u; i += blockDim.x) dst[i] = src[i];
}

// Host side of one persistent launch over a set of populations.
struct PersistBatch {
    void *d_sir = nullptr, *d_wealth = nullptr, *d_walk = nullptr, *d_queue = nullptr;
    uint32_t *d_codes = nullptr, *d_claimed = nullptr, *d_done = nullptr, *d_ctl = nullptr, *wide = nullptr;
    const uint32_t **d_tinf = nullptr;
    uint32_t *d_K = nullptr;
    PersistArgs args{};
    uint32_t grid = 0, n_sir = 0;
    size_t smem = 0;
    std::vector<amb_pop *> sir_pops;
    std::vector<uint32_t> sir_steps;

    void release(cudaStream_t s)
    {
        dfree(d_sir, s);
        dfree(d_wealth, s);
        dfree(d_walk, s);
        dfree(d_queue, s);
        dfree(d_codes, s);
        dfree(d_claimed, s);
        dfree(d_done, s);
        dfree(d_ctl, s);
        dfree(wide, s);
        void *t = const_cast<uint32_t **>(d_tinf);
        dfree(t, s);
        d_tinf = nullptr;
        dfree(d_K, s);
    }
};

static amb_status persist_build(PersistBatch &pb, const std::vector<amb_pop *> &pops, const std::vector<uint32_t> &ks,
                                BandShape shape, cudaStream_t s, uint32_t *units_out)
{
    const uint32_t sms = device_sms();
    std::vector<SirJob> sir;
    std::vector<WealthJob> wealth;
    std::vector<WalkJob> walk;
    std::vector<QEntry> queue;
    std::vector<const uint32_t *> tinf;
    std::vector<uint32_t> Ks;
    uint64_t n_entries = 0, units = 0;
    size_t smem = 16, wide_words = 0;
    // the counters of a band share the CTA's shared memory with the kernel's
    // static tables
    static uint32_t static_smem = 0;
    if (!static_smem) {
        cudaFuncAttributes fa;
        AMB_TRY_CUDA(cudaFuncGetAttributes(&fa, persist_kernel));
        static_smem = (uint32_t)fa.sharedSizeBytes;
    }
    int optin = 0, dev = 0;
    AMB_TRY_CUDA(cudaGetDevice(&dev));
    AMB_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    shape.smem_cap = (uint32_t)std::max<int>(0, optin - (int)static_smem - 160);
    if (shape.adaptive) {
        uint64_t fewest = 0;
        for (size_t i = 0; i < pops.size(); ++i)
            if (pops[i]->model == AMB_SIR && ks[i] && pops[i]->p.n)
                fewest += sir_fewest_bands(pops[i]->p.grid_side, shape.rows_cap, shape.smem_cap);
        shape.spread = fewest < 2ull * sms;
    }
    for (size_t i = 0; i < pops.size(); ++i) {
        amb_pop *p = pops[i];
        const uint32_t k = ks[i];
        if (k == 0 || p->p.n == 0) continue;
        if (p->model == AMB_SIR) {
            AMB_TRY(sir_band_regeometry(p, shape));
            SirJob j;
            memset(&j, 0, sizeof(j));
            BandArgs &a = j.a;
            const int in = p->cur, out = p->cur ^ 1;
            a.rec_in = p->rec[in];
            a.row_in = p->row_start[in];
            a.rec_out = p->rec[out];
            a.row_out = p->row_start[out];
            a.start = p->start;
            a.n = p->p.n;
            a.L = p->p.grid_side;
            a.H = p->band_rows;
            a.n_bands = p->n_bands;
            a.k0 = p->key0;
            a.k1 = p->key1;
            a.t = (uint32_t)p->t;
            a.t_inf = p->t_inf_d;
            a.K = p->K;
            a.t_rec = p->t_rec;
            a.row = p->series + (size_t)p->t * 4u;
            a.status = p->lb.status;
            a.err = p->err;
            j.t_end = (uint32_t)(p->t + k);
            // epochs of this run's steps continue the population's own launches
            j.epoch_base = p->lb.launches - (uint32_t)p->t;
            a.code_tab = nullptr;
            queue.push_back(QEntry{kKindSir, (uint32_t)sir.size(), p->n_bands, 1u});
            n_entries += k;
            units += p->n_bands;
            sir.push_back(j);
            tinf.push_back(p->t_inf_d);
            Ks.push_back(p->K);
            pb.sir_pops.push_back(p);
            pb.sir_steps.push_back(k);
            smem = std::max<size_t>(smem, p->band_smem);
            if (p->p.n >= kPackedLimit) wide_words = std::max<size_t>(wide_words, (size_t)2u * p->band_rows * a.L);
        } else if (p->model == AMB_WEALTH) {
            WealthJob w;
            memset(&w, 0, sizeof(w));
            w.w = p->w;
            w.credit = p->credit;
            w.series = p->series;
            w.n = p->p.n;
            w.k0 = p->key0;
            w.k1 = p->key1;
            w.t = (uint32_t)p->t;
            w.t_end = (uint32_t)(p->t + k);
            if (wealth_uses_smem(p->p.n)) {
                queue.push_back(QEntry{kKindWealthSmall, (uint32_t)wealth.size(), 1u, 1u});
                n_entries += 1;
                units += 1;
                smem = std::max<size_t>(smem, (size_t)((p->p.n + 7u) & ~7u) * 4u + (size_t)p->p.n * 2u + 16u);
            } else {
                const uint32_t c = (p->p.n + kUnitAgents - 1u) / kUnitAgents;
                queue.push_back(QEntry{kKindDonate, (uint32_t)wealth.size(), c, 1u});
                n_entries += 2ull * k;
                units += c;
            }
            wealth.push_back(w);
        } else {
            WalkJob w;
            memset(&w, 0, sizeof(w));
            w.x = p->x;
            w.y = p->y;
            w.rows = p->series + (size_t)p->t * 4u;
            w.err = p->err;
            w.n = p->p.n;
            w.L = p->p.grid_side;
            w.k0 = p->key0;
            w.k1 = p->key1;
            w.t0 = (uint32_t)p->t;
            w.k = k;
            const uint32_t c = (p->p.n + kUnitAgents - 1u) / kUnitAgents;
            queue.push_back(QEntry{kKindWalk, (uint32_t)walk.size(), c, 1u});
            n_entries += 1;
            units += c;
            walk.push_back(w);
        }
    }
    if (n_entries >= 0x7FFFFFFFull) return fail(AMB_EINVAL, "too many steps in one batch (%llu queue entries)",
                                                (unsigned long long)n_entries);
    const size_t E = std::max<size_t>((size_t)n_entries, 1u);
    pb.n_sir = (uint32_t)sir.size();
    pb.smem = smem;
    pb.grid = (uint32_t)std::max<uint64_t>(1u, std::min<uint64_t>(units, sms));
    if (units_out) *units_out = (uint32_t)std::min<uint64_t>(units, 0xFFFFFFFFu);
    AMB_TRY(dalloc(reinterpret_cast<unsigned char **>(&pb.d_sir), std::max<size_t>(sir.size(), 1) * sizeof(SirJob), s));
    AMB_TRY(dalloc(reinterpret_cast<unsigned char **>(&pb.d_wealth), std::max<size_t>(wealth.size(), 1) * sizeof(WealthJob), s));
    AMB_TRY(dalloc(reinterpret_cast<unsigned char **>(&pb.d_walk), std::max<size_t>(walk.size(), 1) * sizeof(WalkJob), s));
    AMB_TRY(dalloc(reinterpret_cast<unsigned char **>(&pb.d_queue), E * sizeof(QEntry), s));
    AMB_TRY(dalloc(&pb.d_claimed, E, s));
    AMB_TRY(dalloc(&pb.d_done, E, s));
    AMB_TRY(dalloc(&pb.d_ctl, 4, s));
    AMB_TRY(dalloc(&pb.d_codes, std::max<size_t>(sir.size(), 1) * kCodeWords, s));
    AMB_TRY(dalloc(reinterpret_cast<const uint32_t ***>(&pb.d_tinf), std::max<size_t>(sir.size(), 1), s));
    AMB_TRY(dalloc(&pb.d_K, std::max<size_t>(sir.size(), 1), s));
    if (wide_words) AMB_TRY(dalloc(&pb.wide, (size_t)pb.grid * wide_words, s));
    AMB_TRY_CUDA(cudaMemsetAsync(pb.d_queue, 0, E * sizeof(QEntry), s));
    AMB_TRY_CUDA(cudaMemsetAsync(pb.d_claimed, 0, E * sizeof(uint32_t), s));
    AMB_TRY_CUDA(cudaMemsetAsync(pb.d_done, 0, E * sizeof(uint32_t), s));
    const uint32_t ctl[4] = {0u, (uint32_t)queue.size(), 0u, 0u};
    AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
    if (!queue.empty())
        AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_queue, queue.data(), queue.size() * sizeof(QEntry), cudaMemcpyHostToDevice, s));
    if (!sir.empty()) {
        AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_sir, sir.data(), sir.size() * sizeof(SirJob), cudaMemcpyHostToDevice, s));
        AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_tinf, tinf.data(), tinf.size() * sizeof(uint32_t *), cudaMemcpyHostToDevice, s));
        AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_K, Ks.data(), Ks.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        code_tables_kernel<<<(unsigned)sir.size(), 256, 0, s>>>(pb.d_tinf, pb.d_K, pb.d_codes);
        AMB_TRY_CUDA(cudaGetLastError());
    }
    if (!wealth.empty())
        AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_wealth, wealth.data(), wealth.size() * sizeof(WealthJob), cudaMemcpyHostToDevice, s));
    if (!walk.empty())
        AMB_TRY_CUDA(cudaMemcpyAsync(pb.d_walk, walk.data(), walk.size() * sizeof(WalkJob), cudaMemcpyHostToDevice, s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));  // the host tables go out of scope
    PersistArgs &pa = pb.args;
    pa.sir = static_cast<SirJob *>(pb.d_sir);
    pa.wealth = static_cast<WealthJob *>(pb.d_wealth);
    pa.walk = static_cast<WalkJob *>(pb.d_walk);
    pa.codes = pb.d_codes;
    pa.queue = static_cast<QEntry *>(pb.d_queue);
    pa.claimed = pb.d_claimed;
    pa.done = pb.d_done;
    pa.ctl = pb.d_ctl;
    pa.n_entries = (uint32_t)n_entries;
    pa.wide = pb.wide;
    pa.wide_words = (uint32_t)wide_words;
    // the kernel may take as much dynamic shared memory as the device allows
    // (set once, to the largest value: every launch asks for its own size)
    static bool attr_set = false;
    if (!attr_set) {
        AMB_TRY_CUDA(cudaFuncSetAttribute(persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          optin - (int)static_smem));
        attr_set = true;
    }
    if (pb.smem > (size_t)(optin - (int)static_smem))
        return fail(AMB_EINVAL, "a batch needs %zu bytes of shared memory per CTA", pb.smem);
    return AMB_OK;
}

static amb_status persist_launch(PersistBatch &pb, cudaStream_t s, uint64_t *launches)
{
    if (pb.args.n_entries == 0) return AMB_OK;
    persist_kernel<<<pb.grid, kBandNT, pb.smem, s>>>(pb.args);
    AMB_TRY_CUDA(cudaGetLastError());
    *launches += 1;
    return AMB_OK;
}

// After the launch: the populations' host-side step counters, buffer parity
// and look-back epochs continue after the run.
static void persist_finish(PersistBatch &pb)
{
    for (size_t q = 0; q < pb.sir_pops.size(); ++q) {
        amb_pop *p = pb.sir_pops[q];
        const uint32_t k = pb.sir_steps[q];
        if (k & 1u) p->cur ^= 1;
        // later epochs must exceed the run's, and a single-population launch
        // must keep the parity its ticket counters expect (the counter of the
        // parity it used last is the one not reset): lb.launches advances by
        // an even number
        p->lb.launches += k + (k & 1u);
    }
}

// Advance every population by its own number of steps (ks[i] for pops[i]) in
// at most three persistent launches (captured as one CUDA graph with graph).
// *ms: device time of the launches (events on s).  Returns after the work is
// done.
amb_status advance(const std::vector<amb_pop *> &pops, const std::vector<uint32_t> &ks, BandShape shape,
                   cudaStream_t s, bool graph, uint64_t *launches_out, float *ms_out)
{
    for (size_t i = 0; i < pops.size(); ++i) {
        amb_pop *p = pops[i];
        const uint32_t k = ks[i];
        if (p->t + k >= (uint64_t)kInitStep) return fail(AMB_EINVAL, "job %zu: too many steps", i);
        AMB_TRY(band_sync_records(p));
        AMB_TRY(ensure_series(p, p->t + k));
        if (k) AMB_TRY_CUDA(cudaMemsetAsync(p->series + (size_t)p->t * 4u, 0, (size_t)k * 4u * sizeof(int64_t), s));
        p->series_next_zero = false;
    }
    // up to three persistent launches, one after the other, by the shared
    // memory their CTAs need: the SIR jobs (band counters), the small wealth
    // jobs (their columns), the large wealth and walk jobs (none).  A launch
    // takes the largest shared memory of its jobs, and the L1 left beside it
    // then limits the memory requests in flight of the large wealth jobs'
    // phases: small and large wealth jobs in one launch took 290 ms on the
    // 1,024-job sweep, apart 159 ms.
    constexpr int kGroups = 3;
    std::vector<amb_pop *> gp[kGroups];
    std::vector<uint32_t> gk[kGroups];
    for (size_t i = 0; i < pops.size(); ++i) {
        const amb_pop *p = pops[i];
        const int g = p->model == AMB_SIR ? 0 : (p->model == AMB_WEALTH && wealth_uses_smem(p->p.n) ? 1 : 2);
        gp[g].push_back(pops[i]);
        gk[g].push_back(ks[i]);
    }
    PersistBatch pb[kGroups];
    amb_status r = AMB_OK;
    for (int g = 0; g < kGroups && r == AMB_OK; ++g) r = persist_build(pb[g], gp[g], gk[g], shape, s, nullptr);
    cudaGraph_t gr = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint64_t launches = 0;
    auto issue = [&]() -> amb_status {
        for (int g = 0; g < kGroups; ++g) AMB_TRY(persist_launch(pb[g], s, &launches));
        return AMB_OK;
    };
    if (r == AMB_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        r = fail(AMB_ECUDA, "event creation failed");
    if (r == AMB_OK && graph) {
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            r = fail(AMB_ECUDA, "stream capture failed to begin (is the stream the legacy default stream?)");
        } else {
            r = issue();
            const cudaError_t ec = cudaStreamEndCapture(s, &gr);
            if (r == AMB_OK && ec != cudaSuccess) r = fail(AMB_ECUDA, "capture: %s", cudaGetErrorString(ec));
            if (r == AMB_OK && cudaGraphInstantiate(&ge, gr, 0) != cudaSuccess) r = fail(AMB_ECUDA, "graph instantiate failed");
        }
        if (r == AMB_OK) {
            cudaEventRecord(e0, s);
            if (cudaGraphLaunch(ge, s) != cudaSuccess) r = fail(AMB_ECUDA, "graph launch failed");
            cudaEventRecord(e1, s);
        }
    } else if (r == AMB_OK) {
        cudaEventRecord(e0, s);
        r = issue();
        cudaEventRecord(e1, s);
    }
    if (r == AMB_OK) {
        const cudaError_t es = cudaEventSynchronize(e1);
        if (es != cudaSuccess) r = fail(AMB_ECUDA, "batched steps: %s", cudaGetErrorString(es));
        float ms = 0.f;
        if (r == AMB_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) *ms_out = ms;
        uint32_t ctl[kGroups][4] = {};
        for (int g = 0; g < kGroups; ++g)
            if (r == AMB_OK && pb[g].d_ctl &&
                cudaMemcpy(ctl[g], pb[g].d_ctl, sizeof(ctl[g]), cudaMemcpyDeviceToHost) != cudaSuccess)
                r = fail(AMB_ECUDA, "reading the run's status failed");
        // the populations moved on (even if the run reports a problem)
        for (int g = 0; g < kGroups; ++g) persist_finish(pb[g]);
        for (size_t i = 0; i < pops.size(); ++i) {
            amb_pop *p = pops[i];
            p->t += ks[i];
            p->launches += ks[i];
            if (p->model == AMB_WALK) p->index_valid = false;
        }
        if (launches_out) *launches_out += launches;
        for (int g = 0; g < kGroups && r == AMB_OK; ++g) {
            if (ctl[g][2] & ERR_TIMEOUT)
                r = fail(AMB_ETIMEOUT, "the batched launch stopped: a wait for queued work ran out");
            else if (ctl[g][2])
                r = fail(AMB_ECUDA, "the batched launch's work queue overflowed (0x%x)", ctl[g][2]);
            else if (pb[g].args.n_entries && ctl[g][0] < pb[g].args.n_entries)
                r = fail(AMB_ETIMEOUT, "the batched launch ended with %u of %u entries taken", ctl[g][0],
                         pb[g].args.n_entries);
        }
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (gr) cudaGraphDestroy(gr);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int g = 0; g < kGroups; ++g) pb[g].release(s);
    cudaStreamSynchronize(s);
    return r;
}

// The error words of every population (one synchronisation).
amb_status read_errors(const std::vector<amb_pop *> &pops, cudaStream_t s, std::vector<uint32_t> &words)
{
    words.assign(pops.size(), 0u);
    for (size_t i = 0; i < pops.size(); ++i)
        AMB_TRY_CUDA(cudaMemcpyAsync(&words[i], pops[i]->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));
    return AMB_OK;
}

amb_status check_errors(const std::vector<amb_pop *> &pops, cudaStream_t s)
{
    std::vector<uint32_t> h;
    AMB_TRY(read_errors(pops, s, h));
    for (size_t i = 0; i < pops.size(); ++i) {
        if (h[i] & ERR_TIMEOUT) return fail(AMB_ETIMEOUT, "job %zu: a bounded device-side wait ran out (0x%x)", i, h[i]);
        if (h[i]) return fail(AMB_EINVARIANT, "job %zu: device reported an out-of-range value (0x%x)", i, h[i]);
    }
    return AMB_OK;
}

}  // namespace amb

using namespace amb;

struct amb_batch {
    cudaStream_t stream = nullptr;
    std::vector<amb_job> jobs;
    std::vector<amb_pop *> pops;
    bool ran = false;
    BandShape shape;
    uint64_t launches = 0;
    double ms = 0.0;
};

namespace {

void destroy_pops(std::vector<amb_pop *> &pops)
{
    for (amb_pop *p : pops)
        if (p) amb_destroy(p);
    pops.clear();
}

amb_status create_pops(const amb_job *jobs, size_t n, cudaStream_t s, std::vector<amb_pop *> &pops)
{
    pops.assign(n, nullptr);
    for (size_t i = 0; i < n; ++i) {
        amb_params p = jobs[i].params;
        if (jobs[i].model == AMB_SIR) p.variant = AMB_SIR_BAND;
        const amb_status st = amb_create(jobs[i].model, &p, jobs[i].seed, jobs[i].replicate, s, &pops[i]);
        if (st != AMB_OK) {
            destroy_pops(pops);
            return st;
        }
    }
    return AMB_OK;
}

// Batched SIR steps of `pops` with the given band shape: `steps` steps in one
// persistent launch, timed on s.
amb_status time_sir(std::vector<amb_pop *> &pops, uint32_t steps, BandShape shape, cudaStream_t s, float *ms)
{
    std::vector<uint32_t> st(pops.size(), steps);
    uint64_t launches = 0;
    return advance(pops, st, shape, s, false, &launches, ms);
}

// Band shape with the shortest batched SIR steps on throwaway copies of (up
// to) the eight largest SIR jobs: caps of 8, 16 and 32 rows, fewest or spread
// bands.
amb_status autotune_shape(const std::vector<amb_job> &jobs, cudaStream_t s, BandShape *best_shape)
{
    std::vector<size_t> sir;
    for (size_t i = 0; i < jobs.size(); ++i)
        if (jobs[i].model == AMB_SIR && jobs[i].params.n > 0 && jobs[i].steps > 0) sir.push_back(i);
    *best_shape = BandShape{};
    if (sir.empty()) return AMB_OK;
    std::sort(sir.begin(), sir.end(), [&](size_t a, size_t b) { return jobs[a].params.n > jobs[b].params.n; });
    if (sir.size() > 8) sir.resize(8);
    std::vector<amb_job> sample;
    for (size_t i : sir) sample.push_back(jobs[i]);
    float best = 1e30f;
    for (int spread = 0; spread < 2; ++spread) {
        for (uint32_t c : {8u, 16u, 32u}) {
            BandShape shape;
            shape.rows_cap = c;
            shape.spread = spread != 0;
            std::vector<amb_pop *> pops;
            AMB_TRY(create_pops(sample.data(), sample.size(), s, pops));
            float warm = 0.f, ms = 0.f;
            amb_status r = time_sir(pops, 1, shape, s, &warm);
            if (r == AMB_OK) r = time_sir(pops, 3, shape, s, &ms);
            if (r == AMB_OK) r = check_errors(pops, s);
            destroy_pops(pops);
            AMB_TRY(r);
            if (ms < best) {
                best = ms;
                *best_shape = shape;
            }
        }
    }
    return AMB_OK;
}

}  // namespace

extern "C" {

amb_status amb_batch_create(const amb_job *jobs, size_t n, void *cuda_stream, amb_batch **out)
{
    AMB_TRACE("amb_batch_create");
    if (!out || (!jobs && n)) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    for (size_t i = 0; i < n; ++i)
        if (jobs[i].model == AMB_SIR && jobs[i].params.variant == AMB_SIR_GENERIC)
            return fail(AMB_EINVAL, "job %zu: batches run SIR on the band path", i);
    amb_batch *b = new (std::nothrow) amb_batch();
    if (!b) return fail(AMB_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->jobs.assign(jobs, jobs + n);
    const amb_status st = create_pops(jobs, n, b->stream, b->pops);
    if (st != AMB_OK) {
        delete b;
        return st;
    }
    *out = b;
    return AMB_OK;
}

amb_status amb_batch_run(amb_batch *b, const amb_tune *tune, double *ms_out)
{
    AMB_TRACE("amb_batch_run");
    if (!b) return fail(AMB_EINVAL, "null batch");
    if (b->ran) return fail(AMB_EINVAL, "a batch runs once");
    cudaStream_t s = b->stream;
    BandShape shape;
    if (tune && tune->band_rows_cap) shape.rows_cap = std::min<uint32_t>(tune->band_rows_cap, kMaxBandRows);
    shape.spread = tune && tune->spread_bands;
    const bool graph = !tune || tune->use_graph;
    if (tune && tune->autotune) AMB_TRY(autotune_shape(b->jobs, s, &shape));
    b->shape = shape;
    std::vector<uint32_t> ks(b->jobs.size());
    for (size_t i = 0; i < ks.size(); ++i) ks[i] = b->jobs[i].steps;
    uint64_t launches = 0;
    float ms = 0.f;
    AMB_TRY(advance(b->pops, ks, shape, s, graph, &launches, &ms));
    b->ms = ms;
    if (ms_out) *ms_out = ms;
    b->launches = launches;
    b->ran = true;
    return check_errors(b->pops, s);
}

amb_status amb_batch_population(amb_batch *b, size_t i, amb_pop **pop)
{
    if (!b || !pop) return fail(AMB_EINVAL, "null pointer");
    if (i >= b->pops.size()) return fail(AMB_EINVAL, "job %zu out of range", i);
    *pop = b->pops[i];
    return AMB_OK;
}

amb_status amb_batch_info(amb_batch *b, amb_batch_report *info)
{
    if (!b || !info) return fail(AMB_EINVAL, "null pointer");
    info->n_jobs = b->pops.size();
    info->band_rows_cap = b->shape.rows_cap;
    info->spread_bands = b->shape.spread ? 1 : 0;
    info->launches = b->launches;
    info->ms = b->ms;
    uint64_t as = 0;
    for (size_t i = 0; i < b->jobs.size(); ++i) as += (uint64_t)b->jobs[i].params.n * b->jobs[i].steps;
    info->agent_steps = as;
    return AMB_OK;
}

amb_status amb_batch_destroy(amb_batch *b)
{
    if (!b) return AMB_OK;
    destroy_pops(b->pops);
    delete b;
    return AMB_OK;
}

}  // extern "C"
