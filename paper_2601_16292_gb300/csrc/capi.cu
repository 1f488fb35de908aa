// capi.cu -- extern "C" entry points of include/amb.h: argument checks,
// population lifetime, dispatch to the model kernels, read-back, invariants
// and statistics.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "amb_internal.cuh"

namespace amb {

static thread_local char g_err[1024];

amb_status fail(amb_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

void clear_error() { g_err[0] = 0; }

unsigned device_sms()
{
    constexpr int kMaxDevices = 64;
    static std::atomic<unsigned> cache[kMaxDevices];  // 0 = not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = -1;
    if (dev >= 0) {
        const unsigned c = cache[dev].load(std::memory_order_relaxed);
        if (c) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev) != cudaSuccess || sms < 1)
        sms = 1;
    if (dev >= 0) cache[dev].store((unsigned)sms, std::memory_order_relaxed);
    return (unsigned)sms;
}

// ------------------------------------------------------------ thresholds ---
// Probability -> uint32 threshold: an event of probability p happens iff the
// uniform 32-bit word is below min(floor(p * 2^32), 2^32 - 1).
static uint32_t threshold_of(double p)
{
    const double scaled = p * 4294967296.0;  // exact: multiplication by 2^32
    if (!(scaled > 0.0)) return 0u;
    if (scaled >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)scaled;
}

amb_status host_thresholds(double beta, double gamma, uint32_t cap, uint32_t *t_inf, uint32_t *K, uint32_t *t_rec)
{
    if (!(beta >= 0.0 && beta <= 1.0)) return fail(AMB_EINVAL, "beta must be in [0, 1]");
    if (!(gamma >= 0.0 && gamma <= 1.0)) return fail(AMB_EINVAL, "gamma must be in [0, 1]");
    if (cap < 1) cap = 1;
    // escape probability after k infected cell-mates, one IEEE product per k
    const double miss = 1.0 - beta;
    double escape = 1.0;
    t_inf[0] = 0u;
    uint32_t last = cap;
    for (uint32_t k = 1; k <= cap; ++k) {
        const double escape_k = escape * miss;
        const double hit = 1.0 - escape_k;
        t_inf[k] = threshold_of(hit);
        if (t_inf[k] == 0xFFFFFFFFu) {
            last = k;
            break;
        }
        if (escape_k == escape) {  // the power is stuck: every later entry is equal
            last = k > 1 ? k - 1 : 1;
            break;
        }
        escape = escape_k;
    }
    *K = last;
    *t_rec = threshold_of(gamma);
    return AMB_OK;
}

// ---------------------------------------------------- launchers elsewhere ---
amb_status walk_steps(amb_pop *pop, uint32_t k);
amb_status wealth_steps(amb_pop *pop, uint32_t k);
bool wealth_uses_smem(uint32_t n);
amb_status sir_generic_steps(amb_pop *pop, uint32_t k);
amb_status sir_band_init(amb_pop *pop, const int32_t *x, const int32_t *y, const uint8_t *state);
amb_status sir_band_steps(amb_pop *pop, uint32_t k);
amb_status sir_band_read(amb_pop *pop, amb_col col, void *dst_dev);
amb_status sir_band_occupancy(amb_pop *pop, int32_t *occ);
bool sir_band_supported(uint32_t L, uint32_t *band_rows);
void sir_band_release(amb_pop *pop);
amb_status launch_minmax_sum(const int32_t *v, uint32_t n, int32_t *mm, unsigned long long *sum, cudaStream_t s);
amb_status launch_value_hist(const int32_t *v, uint32_t n, int32_t base, uint32_t bins, unsigned long long *hist,
                             cudaStream_t s);
amb_status launch_gini_numerator(const unsigned long long *hist, uint32_t bins, int32_t base, uint32_t n,
                                 long long *out, cudaStream_t s);
amb_status launch_occupancy(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *occ, cudaStream_t s);
amb_status launch_occupancy_from_start(const int32_t *start, uint64_t C, int32_t *occ, cudaStream_t s);
amb_status launch_max(const int32_t *v, uint64_t m, int32_t *out, cudaStream_t s);
amb_status launch_count_hist(const int32_t *v, uint64_t m, uint32_t bins, unsigned long long *hist, cudaStream_t s);
amb_status launch_curve_sums(const int64_t *series, uint32_t T, long long *out, cudaStream_t s);
amb_status launch_bounds_check(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, unsigned long long *bad,
                               cudaStream_t s);
amb_status launch_monotone_check(const int32_t *start, uint64_t C, unsigned long long *bad, cudaStream_t s);
amb_status launch_state_count(const uint8_t *st, uint32_t n, unsigned long long *cnt, cudaStream_t s);

// ------------------------------------------------------------ init kernels ---
__global__ void init_positions_kernel(int32_t *__restrict__ x, int32_t *__restrict__ y, uint32_t n, uint32_t L,
                                      uint32_t k0, uint32_t k1)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const U4 u = philox(i, kInitStep, k0, k1);
        x[i] = (int32_t)below(u.w0, L);
        y[i] = (int32_t)below(u.w1, L);
    }
}

__global__ void init_state_kernel(uint8_t *__restrict__ st, uint32_t n, uint32_t n0)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        st[i] = (uint8_t)(i < n0 ? AMB_I : AMB_S);
}

__global__ void fill_i32_kernel(int32_t *__restrict__ v, uint32_t n, int32_t val)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = val;
}

// counts values outside [0, hi) (int32) -> bad
__global__ void range_check_i32_kernel(const int32_t *__restrict__ v, uint32_t n, uint32_t hi,
                                       unsigned long long *__restrict__ bad)
{
    uint32_t b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        b += ((uint32_t)v[i] >= hi);
    if (b) atomicAdd(bad, (unsigned long long)b);
}

__global__ void range_check_u8_kernel(const uint8_t *__restrict__ v, uint32_t n, uint32_t hi,
                                      unsigned long long *__restrict__ bad)
{
    uint32_t b = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b += (v[i] >= hi);
    if (b) atomicAdd(bad, (unsigned long long)b);
}

// ------------------------------------------------------------ helpers ---
// Orders the population's stream after the counts copies queued on the side
// stream (the last copy event covers the earlier ones: the side stream is in
// order).
static amb_status join_copies(amb_pop *pop)
{
    if (!pop->copies_pending) return AMB_OK;
    AMB_TRY_CUDA(cudaStreamWaitEvent(pop->stream, pop->ev_copied, 0));
    pop->copies_pending = false;
    return AMB_OK;
}

static amb_status device_error(amb_pop *pop)
{
    AMB_TRY(join_copies(pop));
    uint32_t h = 0;
    AMB_TRY_CUDA(cudaMemcpyAsync(&h, pop->err, sizeof(h), cudaMemcpyDeviceToHost, pop->stream));
    AMB_TRY_CUDA(cudaStreamSynchronize(pop->stream));
    if (h & ERR_TIMEOUT) return fail(AMB_ETIMEOUT, "a bounded device-side wait ran out (error word 0x%x)", h);
    if (h & (ERR_RANGE | ERR_OVERFLOW))
        return fail(AMB_EINVARIANT, "device reported an out-of-range value (error word 0x%x)", h);
    return AMB_OK;
}

amb_status ensure_series(amb_pop *pop, uint64_t rows)
{
    if (rows <= pop->series_cap) return AMB_OK;
    size_t cap = pop->series_cap ? pop->series_cap : 64;
    while (cap < rows) cap *= 2;
    int64_t *ns = nullptr;
    AMB_TRY(dalloc(&ns, cap * 4u, pop->stream));
    if (pop->series && pop->t)
        AMB_TRY_CUDA(cudaMemcpyAsync(ns, pop->series, (size_t)pop->t * 4u * sizeof(int64_t), cudaMemcpyDeviceToDevice,
                                     pop->stream));
    AMB_TRY(join_copies(pop));  // pending copies still read the old rows
    dfree(pop->series, pop->stream);
    pop->series = ns;
    pop->series_cap = cap;
    pop->series_next_zero = false;
    return AMB_OK;
}

static amb_status count_bad_i32(amb_pop *pop, const int32_t *v, uint32_t n, uint32_t hi, unsigned long long *h)
{
    unsigned long long *bad = nullptr;
    AMB_TRY(dalloc(&bad, 1, pop->stream));
    cudaMemsetAsync(bad, 0, sizeof(*bad), pop->stream);
    if (n) range_check_i32_kernel<<<grid_for(n, 256, 8u), 256, 0, pop->stream>>>(v, n, hi, bad);
    cudaMemcpyAsync(h, bad, sizeof(*h), cudaMemcpyDeviceToHost, pop->stream);
    dfree(bad, pop->stream);
    AMB_TRY_CUDA(cudaStreamSynchronize(pop->stream));
    return AMB_OK;
}

static amb_status count_bad_u8(amb_pop *pop, const uint8_t *v, uint32_t n, uint32_t hi, unsigned long long *h)
{
    unsigned long long *bad = nullptr;
    AMB_TRY(dalloc(&bad, 1, pop->stream));
    cudaMemsetAsync(bad, 0, sizeof(*bad), pop->stream);
    if (n) range_check_u8_kernel<<<grid_for(n, 256, 8u), 256, 0, pop->stream>>>(v, n, hi, bad);
    cudaMemcpyAsync(h, bad, sizeof(*h), cudaMemcpyDeviceToHost, pop->stream);
    dfree(bad, pop->stream);
    AMB_TRY_CUDA(cudaStreamSynchronize(pop->stream));
    return AMB_OK;
}

static amb_status copy_out(const void *src_dev, void *dst, size_t bytes, int dst_on_device, cudaStream_t s)
{
    if (bytes == 0) return AMB_OK;
    AMB_TRY_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));
    return AMB_OK;
}

static bool uses_band(const amb_pop *pop) { return pop->model == AMB_SIR && pop->path == AMB_SIR_BAND; }

// Band path after column writes: rebuild the cell-ordered records from the
// staged id-ordered columns (once, however many columns were written).
amb_status band_sync_records(amb_pop *pop)
{
    if (!uses_band(pop) || !pop->band_dirty) return AMB_OK;
    cudaStream_t s = pop->stream;
    const amb_status st = sir_band_init(pop, pop->x, pop->y, pop->state);
    dfree(pop->x, s);
    dfree(pop->y, s);
    dfree(pop->state, s);
    pop->band_dirty = false;
    return st;
}

// Cell index of the current positions for the id-ordered layouts.
static amb_status build_index(amb_pop *pop)
{
    const uint32_t n = pop->p.n, L = pop->p.grid_side;
    const uint64_t C = (uint64_t)L * L;
    if (!pop->start) AMB_TRY(dalloc(&pop->start, C + 1, pop->stream));
    if (!pop->ids) AMB_TRY(dalloc(&pop->ids, n, pop->stream));
    int32_t *cnt = pop->cnt, *cursor = pop->cursor;
    bool tmp = false;
    if (!cnt || !cursor) {
        AMB_TRY(dalloc(&cnt, C, pop->stream));
        AMB_TRY(dalloc(&cursor, C, pop->stream));
        tmp = true;
    }
    amb_status st = launch_cell_index(pop->x, pop->y, n, L, pop->start, pop->ids, cnt, cursor, pop->lb, pop->err,
                                      pop->stream);
    if (tmp) {
        dfree(cnt, pop->stream);
        dfree(cursor, pop->stream);
    }
    if (st == AMB_OK) pop->index_valid = true;
    return st;
}

static void release(amb_pop *pop)
{
    cudaStream_t s = pop->stream;
    join_copies(pop);
    dfree(pop->w, s);
    dfree(pop->credit, s);
    dfree(pop->x, s);
    dfree(pop->y, s);
    dfree(pop->state, s);
    dfree(pop->cnt, s);
    dfree(pop->inf, s);
    dfree(pop->cursor, s);
    dfree(pop->start, s);
    dfree(pop->ids, s);
    sir_band_release(pop);
    cont_release(pop);
    dfree(pop->t_inf_d, s);
    dfree(pop->series, s);
    dfree(pop->err, s);
    pop->lb.release(s);
}

}  // namespace amb

using namespace amb;

extern "C" {

const char *amb_last_error(void) { return g_err; }

const char *amb_version(void) { return "amb 0.1 (sm_103a)"; }

amb_status amb_sir_thresholds(double beta, double gamma, uint32_t cap, uint32_t *t_inf, uint32_t *K, uint32_t *t_rec)
{
    if (!t_inf || !K || !t_rec) return fail(AMB_EINVAL, "null pointer");
    return host_thresholds(beta, gamma, cap, t_inf, K, t_rec);
}

}  // extern "C"

namespace amb {
static std::atomic<uint32_t> g_fail_creates{0};

// consume one injected creation failure, if any are armed
bool injected_create_failure()
{
    uint32_t k = g_fail_creates.load();
    while (k > 0)
        if (g_fail_creates.compare_exchange_weak(k, k - 1)) return true;
    return false;
}

cudaMemPool_t library_pool()
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool tried[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!tried[dev]) {
        tried[dev] = true;
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = p;
        } else {
            (void)cudaGetLastError();
        }
    }
    return pools[dev];
}

// The checks amb_create makes on its arguments (no GPU call).
amb_status check_params(amb_model model, const amb_params *p, uint64_t seed)
{
    if (!p) return fail(AMB_EINVAL, "null pointer");
    if (model == AMB_CWALK || model == AMB_CSIR)
        return fail(AMB_EINVAL, "continuous-space models are created by amb_create_continuous (and are not batched)");
    if (model != AMB_WEALTH && model != AMB_WALK && model != AMB_SIR) return fail(AMB_EINVAL, "unknown model %d", (int)model);
    if (seed > 0xFFFFFFFFull) return fail(AMB_EINVAL, "seed must be < 2^32");
    if (p->n > 0x7FFFFFFFu) return fail(AMB_EINVAL, "n must be < 2^31");
    const uint32_t L = p->grid_side;
    if (model != AMB_WEALTH) {
        if (L < 1 || L > 0x7FFFFFFFu) return fail(AMB_EINVAL, "grid_side must be in [1, 2^31 - 1]");
        if (model == AMB_SIR && (uint64_t)L * L >= 0x80000000ull) return fail(AMB_EINVAL, "SIR needs L*L < 2^31");
    }
    if (model == AMB_SIR) {
        if (!(p->beta >= 0.0 && p->beta <= 1.0) || !(p->gamma >= 0.0 && p->gamma <= 1.0))
            return fail(AMB_EINVAL, "beta and gamma must be in [0, 1]");
        if (p->n_init_infected > p->n) return fail(AMB_EINVAL, "n_init_infected > n");
        if (p->variant > AMB_SIR_BAND16) return fail(AMB_EINVAL, "unknown SIR variant %u", p->variant);
        if (p->variant == AMB_SIR_BAND16 && (L % 8u != 0 || L > 8192u))
            return fail(AMB_EINVAL, "16-bit band counters need L a multiple of 8, at most 8192 (L = %u)", L);
    }
    return AMB_OK;
}

amb_status check_cparams(amb_model model, const amb_cparams *p, uint64_t seed)
{
    if (!p) return fail(AMB_EINVAL, "null pointer");
    if (model != AMB_CWALK && model != AMB_CSIR) return fail(AMB_EINVAL, "not a continuous-space model: %d", (int)model);
    if (seed > 0xFFFFFFFFull) return fail(AMB_EINVAL, "seed must be < 2^32");
    if (p->n > 0x7FFFFFFFu) return fail(AMB_EINVAL, "n must be < 2^31");
    const float lim = 3.0e38f;
    if (!(p->width >= 0.0f && p->width <= lim) || !(p->height >= 0.0f && p->height <= lim))
        return fail(AMB_EINVAL, "the box must have finite sides >= 0");
    if (!(p->step >= 0.0f && p->step <= lim)) return fail(AMB_EINVAL, "step must be finite and >= 0");
    if (model == AMB_CSIR) {
        if (!(p->radius >= 0.0f && p->radius <= lim)) return fail(AMB_EINVAL, "radius must be finite and >= 0");
        if (!(p->p_infect >= 0.0 && p->p_infect <= 1.0)) return fail(AMB_EINVAL, "p_infect must be in [0, 1]");
        if (p->recovery_steps < 1) return fail(AMB_EINVAL, "recovery_steps must be >= 1");
        if (p->n_init_infected > p->n) return fail(AMB_EINVAL, "n_init_infected > n");
    }
    return AMB_OK;
}
}  // namespace amb

extern "C" {

amb_status amb_create(amb_model model, const amb_params *p, uint64_t seed, uint32_t replicate, void *cuda_stream,
                      amb_pop **out)
{
    AMB_TRACE("amb_create");
    if (!p || !out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    AMB_TRY(check_params(model, p, seed));
    if (injected_create_failure()) return fail(AMB_ENOMEM, "injected creation failure");
    const uint32_t L = p->grid_side;
    amb_pop *pop = new (std::nothrow) amb_pop();
    if (!pop) return fail(AMB_ENOMEM, "host allocation failed");
    pop->model = model;
    pop->p = *p;
    pop->key0 = (uint32_t)seed;
    pop->key1 = replicate;
    pop->stream = (cudaStream_t)cuda_stream;
    cudaStream_t s = pop->stream;
    const uint32_t n = p->n;
    amb_status st = AMB_OK;
#define CREATE_TRY(expr)                 \
    do {                                 \
        st = (expr);                     \
        if (st != AMB_OK) goto failed;   \
    } while (0)
#define CREATE_CUDA(call)                                                                              \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            st = fail(AMB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));                      \
            goto failed;                                                                               \
        }                                                                                              \
    } while (0)
    {
        CREATE_TRY(dalloc(&pop->err, 1, s));
        CREATE_CUDA(cudaMemsetAsync(pop->err, 0, sizeof(uint32_t), s));
        CREATE_TRY(ensure_series(pop, 64));
        const unsigned g = grid_for(n, 256, 16u);
        if (model == AMB_WEALTH) {
            CREATE_TRY(dalloc(&pop->w, n, s));
            if (n) fill_i32_kernel<<<g, 256, 0, s>>>(pop->w, n, p->w_init);
            if (!wealth_uses_smem(n)) {
                CREATE_TRY(dalloc(&pop->credit, n, s));
                CREATE_CUDA(cudaMemsetAsync(pop->credit, 0, (size_t)n * sizeof(int32_t), s));
            }
            pop->ref_total = (int64_t)n * (int64_t)p->w_init;
            pop->ref_total_valid = true;
        } else {
            CREATE_TRY(dalloc(&pop->x, n, s));
            CREATE_TRY(dalloc(&pop->y, n, s));
            if (n) init_positions_kernel<<<g, 256, 0, s>>>(pop->x, pop->y, n, L, pop->key0, pop->key1);
            if (model == AMB_SIR) {
                const uint64_t C = (uint64_t)L * L;
                CREATE_TRY(dalloc(&pop->state, n, s));
                if (n) init_state_kernel<<<g, 256, 0, s>>>(pop->state, n, p->n_init_infected);
                // thresholds (host), uploaded once
                const uint32_t cap = n > 0 ? n : 1;
                pop->t_inf_h.assign((size_t)cap + 1, 0u);
                CREATE_TRY(host_thresholds(p->beta, p->gamma, cap, pop->t_inf_h.data(), &pop->K, &pop->t_rec));
                pop->t_inf_h.resize((size_t)pop->K + 1);
                CREATE_TRY(dalloc(&pop->t_inf_d, pop->t_inf_h.size(), s));
                CREATE_CUDA(cudaMemcpyAsync(pop->t_inf_d, pop->t_inf_h.data(), pop->t_inf_h.size() * sizeof(uint32_t),
                                            cudaMemcpyHostToDevice, s));
                pop->init_infected = p->n_init_infected;
                uint32_t band_rows = 0;
                const bool band_ok = sir_band_supported(L, &band_rows);
                pop->path = (p->variant == AMB_SIR_GENERIC || (p->variant == AMB_SIR_AUTO && !band_ok))
                                ? AMB_SIR_GENERIC
                                : AMB_SIR_BAND;
                if (pop->path == AMB_SIR_BAND && !band_ok) {
                    st = fail(AMB_EINVAL, "the band path needs a smaller grid (L = %u)", L);
                    goto failed;
                }
                if (pop->path == AMB_SIR_GENERIC) {
                    CREATE_TRY(dalloc(&pop->cnt, C, s));
                    CREATE_TRY(dalloc(&pop->inf, C, s));
                    CREATE_TRY(dalloc(&pop->cursor, C, s));
                    CREATE_TRY(build_index(pop));
                } else {
                    CREATE_TRY(sir_band_init(pop, pop->x, pop->y, pop->state));
                    dfree(pop->x, s);
                    dfree(pop->y, s);
                    dfree(pop->state, s);
                }
            }
        }
        CREATE_CUDA(cudaGetLastError());
        CREATE_CUDA(cudaStreamSynchronize(s));
        *out = pop;
        return AMB_OK;
    }
failed:
    release(pop);
    cudaStreamSynchronize(s);
    delete pop;
    return st;
#undef CREATE_TRY
#undef CREATE_CUDA
}

amb_status amb_destroy(amb_pop *pop)
{
    if (!pop) return AMB_OK;
    cudaStream_t s = pop->stream;
    release(pop);
    cudaError_t e = cudaStreamSynchronize(s);
    if (pop->copy_stream) cudaStreamDestroy(pop->copy_stream);
    if (pop->ev_ready) cudaEventDestroy(pop->ev_ready);
    if (pop->ev_copied) cudaEventDestroy(pop->ev_copied);
    delete pop;
    if (e != cudaSuccess) return fail(AMB_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
    return AMB_OK;
}

uint64_t amb_step_index(const amb_pop *pop) { return pop ? pop->t : 0; }

amb_status amb_synchronize(amb_pop *pop)
{
    if (!pop) return fail(AMB_EINVAL, "null population");
    return device_error(pop);
}

amb_status amb_step(amb_pop *pop, uint32_t k)
{
    AMB_TRACE("amb_step");
    if (!pop) return fail(AMB_EINVAL, "null population");
    AMB_TRY(band_sync_records(pop));
    if (k == 0) return AMB_OK;
    if (pop->t + k >= (uint64_t)kInitStep) return fail(AMB_EINVAL, "step counter would reach 2^32 - 1");
    AMB_TRY(ensure_series(pop, pop->t + k));
    amb_status st = AMB_OK;
    switch (pop->model) {
    case AMB_WEALTH: st = wealth_steps(pop, k); break;
    case AMB_WALK:
        st = walk_steps(pop, k);
        pop->index_valid = false;
        break;
    case AMB_SIR:
        if (pop->path == AMB_SIR_BAND) {
            st = sir_band_steps(pop, k);  // sets series_next_zero
        } else {
            st = sir_generic_steps(pop, k);
            pop->series_next_zero = false;
        }
        break;
    case AMB_CWALK:
    case AMB_CSIR: st = cont_steps(pop, k); break;
    }
    if (st == AMB_OK) pop->t += k;
    return st;
}

amb_status amb_set_step(amb_pop *pop, uint64_t t)
{
    AMB_TRACE("amb_set_step");
    if (!pop) return fail(AMB_EINVAL, "null population");
    if (t >= (uint64_t)kInitStep) return fail(AMB_EINVAL, "step index must be < 2^32 - 1");
    AMB_TRY(device_error(pop));
    cudaStream_t s = pop->stream;
    AMB_TRY(ensure_series(pop, t));
    if (t > pop->t)  // rows of steps that were not run here read as zeros
        AMB_TRY_CUDA(cudaMemsetAsync(pop->series + (size_t)pop->t * 4u, 0, (size_t)(t - pop->t) * 4u * sizeof(int64_t), s));
    pop->t = t;
    pop->series_next_zero = false;
    pop->conservation_from = t;
    pop->monotone_from = t;
    amb_status st = AMB_OK;
    if (uses_band(pop) && pop->band_dirty) {
        st = band_sync_records(pop);  // the staged columns, with the draws of step t
    } else if (uses_band(pop) && pop->p.n) {
        // the records carry each agent's draws for the next step: redraw them for step t
        const uint32_t n = pop->p.n;
        int32_t *x = nullptr, *y = nullptr;
        uint8_t *state = nullptr;
        if ((st = dalloc(&x, n, s)) == AMB_OK && (st = dalloc(&y, n, s)) == AMB_OK &&
            (st = dalloc(&state, n, s)) == AMB_OK && (st = sir_band_read(pop, AMB_COL_X, x)) == AMB_OK &&
            (st = sir_band_read(pop, AMB_COL_Y, y)) == AMB_OK && (st = sir_band_read(pop, AMB_COL_STATE, state)) == AMB_OK)
            st = sir_band_init(pop, x, y, state);
        dfree(x, s);
        dfree(y, s);
        dfree(state, s);
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st == AMB_OK && e != cudaSuccess) st = fail(AMB_ECUDA, "sync: %s", cudaGetErrorString(e));
    return st;
}

amb_status amb_write_column(amb_pop *pop, amb_col col, const void *src, size_t n, int src_on_device)
{
    AMB_TRACE("amb_write_column");
    if (!pop || (!src && n)) return fail(AMB_EINVAL, "null pointer");
    if (n != pop->p.n) return fail(AMB_EINVAL, "column length %zu != n = %u", n, pop->p.n);
    if (is_continuous(pop)) {
        AMB_TRY(device_error(pop));
        return cont_write_column(pop, col, src, n, src_on_device);
    }
    const bool ok_col = (pop->model == AMB_WEALTH && col == AMB_COL_WEALTH) ||
                        (pop->model == AMB_WALK && (col == AMB_COL_X || col == AMB_COL_Y)) ||
                        (pop->model == AMB_SIR && (col == AMB_COL_X || col == AMB_COL_Y || col == AMB_COL_STATE));
    if (!ok_col) return fail(AMB_EINVAL, "column %d does not belong to this model", (int)col);
    AMB_TRY(device_error(pop));
    cudaStream_t s = pop->stream;
    const size_t esz = (col == AMB_COL_STATE) ? 1 : 4;
    const uint32_t L = pop->p.grid_side;
    // stage into a device buffer, validate, then commit
    void *tmp = nullptr;
    AMB_TRY(dalloc((unsigned char **)&tmp, n * esz, s));
    amb_status st = AMB_OK;
    if (n && cudaMemcpyAsync(tmp, src, n * esz, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s) !=
                 cudaSuccess)
        st = fail(AMB_ECUDA, "column upload failed");
    unsigned long long bad = 0;
    if (st == AMB_OK) {
        if (col == AMB_COL_X || col == AMB_COL_Y)
            st = count_bad_i32(pop, (const int32_t *)tmp, (uint32_t)n, L, &bad);
        else if (col == AMB_COL_STATE)
            st = count_bad_u8(pop, (const uint8_t *)tmp, (uint32_t)n, 3u, &bad);
        if (st == AMB_OK && bad) st = fail(AMB_EINVAL, "%llu values out of range", bad);
    }
    if (st == AMB_OK) {
        if (pop->model == AMB_WEALTH) {
            cudaMemcpyAsync(pop->w, tmp, n * 4, cudaMemcpyDeviceToDevice, s);
            int32_t *mm = nullptr;
            unsigned long long *sum = nullptr;
            if ((st = dalloc(&mm, 2, s)) == AMB_OK && (st = dalloc(&sum, 1, s)) == AMB_OK &&
                (st = launch_minmax_sum(pop->w, (uint32_t)n, mm, sum, s)) == AMB_OK) {
                unsigned long long h = 0;
                cudaMemcpyAsync(&h, sum, sizeof(h), cudaMemcpyDeviceToHost, s);
                if (cudaStreamSynchronize(s) == cudaSuccess) {
                    pop->ref_total = (int64_t)h;
                    pop->ref_total_valid = true;
                    pop->conservation_from = pop->t;
                } else {
                    st = fail(AMB_ECUDA, "sync failed");
                }
            }
            dfree(mm, s);
            dfree(sum, s);
        } else if (uses_band(pop)) {
            // stage id-ordered columns (materialised from the records on the
            // first write); the records are rebuilt once, before they are next used
            if (!pop->band_dirty) {
                if ((st = dalloc(&pop->x, n, s)) == AMB_OK && (st = dalloc(&pop->y, n, s)) == AMB_OK &&
                    (st = dalloc(&pop->state, n, s)) == AMB_OK && (st = sir_band_read(pop, AMB_COL_X, pop->x)) == AMB_OK &&
                    (st = sir_band_read(pop, AMB_COL_Y, pop->y)) == AMB_OK &&
                    (st = sir_band_read(pop, AMB_COL_STATE, pop->state)) == AMB_OK) {
                    pop->band_dirty = true;
                } else {
                    dfree(pop->x, s);
                    dfree(pop->y, s);
                    dfree(pop->state, s);
                }
            }
            if (st == AMB_OK) {
                void *dstc = (col == AMB_COL_X) ? (void *)pop->x : (col == AMB_COL_Y) ? (void *)pop->y : (void *)pop->state;
                cudaMemcpyAsync(dstc, tmp, n * esz, cudaMemcpyDeviceToDevice, s);
            }
            pop->monotone_from = pop->t;
        } else {
            void *dstc = (col == AMB_COL_X) ? (void *)pop->x : (col == AMB_COL_Y) ? (void *)pop->y : (void *)pop->state;
            cudaMemcpyAsync(dstc, tmp, n * esz, cudaMemcpyDeviceToDevice, s);
            if (pop->model == AMB_SIR) {
                pop->monotone_from = pop->t;
                if (col != AMB_COL_STATE) st = build_index(pop);
            } else {
                pop->index_valid = false;
            }
        }
    }
    dfree(tmp, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == AMB_OK && e != cudaSuccess) st = fail(AMB_ECUDA, "sync: %s", cudaGetErrorString(e));
    return st;
}

amb_status amb_read_column(amb_pop *pop, amb_col col, void *dst, size_t n, int dst_on_device)
{
    AMB_TRACE("amb_read_column");
    if (!pop || (!dst && n)) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(band_sync_records(pop));
    if (n != pop->p.n) return fail(AMB_EINVAL, "column length %zu != n = %u", n, pop->p.n);
    if (is_continuous(pop)) {
        AMB_TRY(device_error(pop));
        return cont_read_column(pop, col, dst, n, dst_on_device);
    }
    const bool ok_col = (pop->model == AMB_WEALTH && col == AMB_COL_WEALTH) ||
                        (pop->model == AMB_WALK && (col == AMB_COL_X || col == AMB_COL_Y)) ||
                        (pop->model == AMB_SIR && (col == AMB_COL_X || col == AMB_COL_Y || col == AMB_COL_STATE));
    if (!ok_col) return fail(AMB_EINVAL, "column %d does not belong to this model", (int)col);
    AMB_TRY(device_error(pop));
    const size_t esz = (col == AMB_COL_STATE) ? 1 : 4;
    if (uses_band(pop)) {
        void *tmp = nullptr;
        AMB_TRY(dalloc((unsigned char **)&tmp, n * esz, pop->stream));
        amb_status st = sir_band_read(pop, col, tmp);
        if (st == AMB_OK) st = copy_out(tmp, dst, n * esz, dst_on_device, pop->stream);
        dfree(tmp, pop->stream);
        cudaStreamSynchronize(pop->stream);
        return st;
    }
    const void *srcc = (col == AMB_COL_WEALTH) ? (const void *)pop->w
                       : (col == AMB_COL_X)    ? (const void *)pop->x
                       : (col == AMB_COL_Y)    ? (const void *)pop->y
                                               : (const void *)pop->state;
    return copy_out(srcc, dst, n * esz, dst_on_device, pop->stream);
}

amb_status amb_counts(amb_pop *pop, int64_t *out, size_t cap_rows, size_t *rows_out)
{
    if (!pop || (!out && cap_rows)) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(device_error(pop));
    const size_t rows = (size_t)pop->t;
    if (rows_out) *rows_out = rows;
    const size_t m = rows < cap_rows ? rows : cap_rows;
    return copy_out(pop->series, out, m * 4u * sizeof(int64_t), 0, pop->stream);
}

amb_status amb_counts_range(amb_pop *pop, uint64_t first, size_t n_rows, int64_t *out)
{
    if (!pop || (!out && n_rows)) return fail(AMB_EINVAL, "null pointer");
    if (first + n_rows > pop->t) return fail(AMB_EINVAL, "rows %llu..%llu not recorded yet", (unsigned long long)first,
                                             (unsigned long long)(first + n_rows));
    AMB_TRY(device_error(pop));
    return copy_out(pop->series + first * 4u, out, n_rows * 4u * sizeof(int64_t), 0, pop->stream);
}

amb_status amb_counts_async(amb_pop *pop, uint64_t first, size_t n_rows, int64_t *out)
{
    if (!pop || (!out && n_rows)) return fail(AMB_EINVAL, "null pointer");
    if (first + n_rows > pop->t) return fail(AMB_EINVAL, "rows %llu..%llu not recorded yet", (unsigned long long)first,
                                             (unsigned long long)(first + n_rows));
    if (n_rows == 0) return AMB_OK;
    if (!pop->copy_stream) {
        cudaStream_t cs = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
            if (cs) cudaStreamDestroy(cs);
            if (e0) cudaEventDestroy(e0);
            return fail(AMB_ECUDA, "side stream for asynchronous counts could not be created");
        }
        pop->copy_stream = cs;
        pop->ev_ready = e0;
        pop->ev_copied = e1;
    }
    AMB_TRY_CUDA(cudaEventRecord(pop->ev_ready, pop->stream));
    AMB_TRY_CUDA(cudaStreamWaitEvent(pop->copy_stream, pop->ev_ready, 0));
    AMB_TRY_CUDA(cudaMemcpyAsync(out, pop->series + first * 4u, n_rows * 4u * sizeof(int64_t), cudaMemcpyDefault,
                                 pop->copy_stream));
    AMB_TRY_CUDA(cudaEventRecord(pop->ev_copied, pop->copy_stream));
    pop->copies_pending = true;
    return AMB_OK;
}

uint64_t amb_launch_count(const amb_pop *pop) { return pop ? pop->launches : 0; }

amb_status amb_read_index(amb_pop *pop, int32_t *start, int32_t *ids, int dst_on_device)
{
    if (!pop || !start || (!ids && pop->p.n)) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(band_sync_records(pop));
    if (pop->model == AMB_WEALTH || is_continuous(pop)) return fail(AMB_EINVAL, "this model has no integer grid");
    const uint64_t C = (uint64_t)pop->p.grid_side * pop->p.grid_side;
    if (C >= 0x80000000ull) return fail(AMB_EINVAL, "index needs L*L < 2^31");
    AMB_TRY(device_error(pop));
    if (uses_band(pop)) {
        AMB_TRY(copy_out(pop->start, start, (C + 1) * sizeof(int32_t), dst_on_device, pop->stream));
        // the id list is the id half of the cell-ordered records
        const size_t n = pop->p.n;
        if (n == 0) return AMB_OK;
        int32_t *tmp = nullptr;
        AMB_TRY(dalloc(&tmp, n, pop->stream));
        amb_status st = sir_band_read(pop, (amb_col)-1, tmp);
        if (st == AMB_OK) st = copy_out(tmp, ids, n * sizeof(int32_t), dst_on_device, pop->stream);
        dfree(tmp, pop->stream);
        return st;
    }
    if (!pop->index_valid) AMB_TRY(build_index(pop));
    AMB_TRY(copy_out(pop->start, start, (C + 1) * sizeof(int32_t), dst_on_device, pop->stream));
    AMB_TRY(copy_out(pop->ids, ids, (size_t)pop->p.n * sizeof(int32_t), dst_on_device, pop->stream));
    return device_error(pop);
}

amb_status amb_occupancy(amb_pop *pop, int32_t *occ, int dst_on_device)
{
    AMB_TRACE("amb_occupancy");
    if (!pop || !occ) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(band_sync_records(pop));
    if (pop->model == AMB_WEALTH) return fail(AMB_EINVAL, "the wealth model has no grid");
    const uint64_t C = (uint64_t)pop->p.grid_side * pop->p.grid_side;
    if (C >= 0x80000000ull) return fail(AMB_EINVAL, "occupancy needs L*L < 2^31");
    AMB_TRY(device_error(pop));
    int32_t *tmp = nullptr;
    AMB_TRY(dalloc(&tmp, C, pop->stream));
    amb_status st = uses_band(pop) ? sir_band_occupancy(pop, tmp)
                                   : launch_occupancy(pop->x, pop->y, pop->p.n, pop->p.grid_side, tmp, pop->stream);
    if (st == AMB_OK) st = copy_out(tmp, occ, C * sizeof(int32_t), dst_on_device, pop->stream);
    dfree(tmp, pop->stream);
    cudaStreamSynchronize(pop->stream);
    return st;
}

amb_status amb_invariants(amb_pop *pop, amb_invariant_report *out)
{
    AMB_TRACE("amb_invariants");
    if (!pop || !out) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(band_sync_records(pop));
    AMB_TRY(device_error(pop));
    amb_invariant_report r;
    r.ok = 1;
    r.conservation_ok = r.nonnegative_ok = r.bounds_ok = r.population_ok = 1;
    r.monotone_ok = r.initial_ok = r.index_ok = 1;
    r.first_bad_step = -1;
    cudaStream_t s = pop->stream;
    const uint32_t n = pop->p.n;
    std::vector<int64_t> rows((size_t)pop->t * 4u);
    AMB_TRY(copy_out(pop->series, rows.data(), rows.size() * sizeof(int64_t), 0, s));
    auto bad_step = [&](uint64_t j) {
        if (r.first_bad_step < 0) r.first_bad_step = (int64_t)j;
    };
    if (pop->model == AMB_WEALTH) {
        for (uint64_t j = pop->conservation_from; j < pop->t; ++j)
            if (pop->ref_total_valid && rows[j * 4 + 1] != pop->ref_total) {
                r.conservation_ok = 0;
                bad_step(j);
            }
        int32_t *mm = nullptr;
        unsigned long long *sum = nullptr;
        AMB_TRY(dalloc(&mm, 2, s));
        AMB_TRY(dalloc(&sum, 1, s));
        AMB_TRY(launch_minmax_sum(pop->w, n, mm, sum, s));
        int32_t hmm[2] = {0, 0};
        AMB_TRY(copy_out(mm, hmm, sizeof(hmm), 0, s));
        dfree(mm, s);
        dfree(sum, s);
        if (n && hmm[0] < 0) r.nonnegative_ok = 0;
    } else if (is_continuous(pop)) {
        bool inside = true;
        AMB_TRY(cont_bounds(pop, &inside));
        if (!inside) r.bounds_ok = 0;
    } else {
        unsigned long long *bad = nullptr;
        AMB_TRY(dalloc(&bad, 2, s));
        AMB_TRY_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned long long), s));
        const uint64_t C = (uint64_t)pop->p.grid_side * pop->p.grid_side;
        if (!uses_band(pop)) AMB_TRY(launch_bounds_check(pop->x, pop->y, n, pop->p.grid_side, &bad[0], s));
        const bool have_index = (pop->model == AMB_SIR) && C < 0x80000000ull;
        if (have_index) AMB_TRY(launch_monotone_check(pop->start, C, &bad[1], s));
        unsigned long long hb[2] = {0, 0};
        AMB_TRY(copy_out(bad, hb, sizeof(hb), 0, s));
        dfree(bad, s);
        if (hb[0]) r.bounds_ok = 0;
        if (have_index) {
            int32_t last = 0;
            AMB_TRY(copy_out(pop->start + C, &last, sizeof(last), 0, s));
            if (hb[1] || last != (int32_t)n) r.index_ok = 0;
        }
    }
    if (pop->model == AMB_SIR || pop->model == AMB_CSIR) {
        {
            int64_t prevR = -1;
            for (uint64_t j = pop->monotone_from; j < pop->t; ++j) {
                const int64_t *q = &rows[j * 4];
                if (q[0] + q[1] + q[2] != (int64_t)n) {
                    r.population_ok = 0;
                    bad_step(j);
                }
                if (prevR >= 0 && q[2] < prevR) {
                    r.monotone_ok = 0;
                    bad_step(j);
                }
                prevR = q[2];
            }
            if (pop->init_infected != (int64_t)pop->p.n_init_infected) r.initial_ok = 0;
        }
    }
    r.ok = r.conservation_ok && r.nonnegative_ok && r.bounds_ok && r.population_ok && r.monotone_ok &&
           r.initial_ok && r.index_ok;
    *out = r;
    if (!r.ok) return fail(AMB_EINVARIANT, "invariant check failed (first bad step %lld)", (long long)r.first_bad_step);
    return AMB_OK;
}

amb_status amb_stats_compute(amb_pop *pop, amb_stats *out, int64_t *hist, size_t hist_cap, size_t *hist_len)
{
    AMB_TRACE("amb_stats_compute");
    if (!pop || !out) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(band_sync_records(pop));
    AMB_TRY(device_error(pop));
    amb_stats r;
    memset(&r, 0, sizeof(r));
    cudaStream_t s = pop->stream;
    const uint32_t n = pop->p.n;
    size_t bins_out = 0;
    if (pop->model == AMB_WEALTH) {
        int32_t *mm = nullptr;
        unsigned long long *sum = nullptr;
        AMB_TRY(dalloc(&mm, 2, s));
        AMB_TRY(dalloc(&sum, 1, s));
        AMB_TRY(launch_minmax_sum(pop->w, n, mm, sum, s));
        int32_t hmm[2];
        unsigned long long hs = 0;
        AMB_TRY(copy_out(mm, hmm, sizeof(hmm), 0, s));
        AMB_TRY(copy_out(sum, &hs, sizeof(hs), 0, s));
        dfree(mm, s);
        dfree(sum, s);
        r.total_wealth = (int64_t)hs;
        if (n) {
            r.min_wealth = hmm[0];
            r.max_wealth = hmm[1];
            const uint64_t bins64 = (uint64_t)((int64_t)hmm[1] - (int64_t)hmm[0]) + 1u;
            if (bins64 > (1u << 26)) return fail(AMB_EINVAL, "wealth range too wide for the histogram");
            const uint32_t bins = (uint32_t)bins64;
            unsigned long long *h = nullptr;
            long long *num = nullptr;
            AMB_TRY(dalloc(&h, bins, s));
            AMB_TRY(dalloc(&num, 2, s));
            AMB_TRY(launch_value_hist(pop->w, n, hmm[0], bins, h, s));
            AMB_TRY(launch_gini_numerator(h, bins, hmm[0], n, num, s));
            long long hn[2];
            AMB_TRY(copy_out(num, hn, sizeof(hn), 0, s));
            if (hist && hist_cap) {
                const size_t m = bins < hist_cap ? bins : hist_cap;
                AMB_TRY(copy_out(h, hist, m * sizeof(int64_t), 0, s));
            }
            dfree(h, s);
            dfree(num, s);
            bins_out = bins;
            r.gini_num_hi = hn[0];
            r.gini_num_lo = (uint64_t)hn[1];
            const __int128 numer = ((__int128)hn[0] << 64) | (__int128)(uint64_t)hn[1];
            const __int128 denom = (__int128)n * (__int128)r.total_wealth;
            r.gini = (r.total_wealth == 0) ? 0.0 : (double)numer / (double)denom;
        }
    } else {
        const uint64_t C = (uint64_t)pop->p.grid_side * pop->p.grid_side;
        if (!is_continuous(pop) && C < 0x80000000ull) {
            int32_t *occ = nullptr, *mx = nullptr;
            AMB_TRY(dalloc(&occ, C, s));
            AMB_TRY(dalloc(&mx, 1, s));
            if (uses_band(pop))
                AMB_TRY(sir_band_occupancy(pop, occ));
            else
                AMB_TRY(launch_occupancy(pop->x, pop->y, n, pop->p.grid_side, occ, s));
            AMB_TRY(launch_max(occ, C, mx, s));
            int32_t hmx = 0;
            AMB_TRY(copy_out(mx, &hmx, sizeof(hmx), 0, s));
            r.max_occupancy = hmx;
            const uint32_t bins = (uint32_t)hmx + 1u;
            unsigned long long *h = nullptr;
            AMB_TRY(dalloc(&h, bins, s));
            AMB_TRY(launch_count_hist(occ, C, bins, h, s));
            if (hist && hist_cap) {
                const size_t m = bins < hist_cap ? bins : hist_cap;
                AMB_TRY(copy_out(h, hist, m * sizeof(int64_t), 0, s));
            }
            bins_out = bins;
            dfree(h, s);
            dfree(occ, s);
            dfree(mx, s);
        }
        if (pop->model == AMB_SIR || pop->model == AMB_CSIR) {
            const uint32_t T = (uint32_t)pop->t;
            long long *cs = nullptr;
            AMB_TRY(dalloc(&cs, 8, s));
            AMB_TRY(launch_curve_sums(pop->series, T, cs, s));
            long long h[8];
            AMB_TRY(copy_out(cs, h, sizeof(h), 0, s));
            dfree(cs, s);
            typedef unsigned __int128 u128;
            const u128 s0 = ((u128)(unsigned long long)h[0] << 64) | (unsigned long long)h[1];
            const u128 s1 = ((u128)(unsigned long long)h[2] << 64) | (unsigned long long)h[3];
            const u128 s2 = ((u128)(unsigned long long)h[4] << 64) | (unsigned long long)h[5];
            r.peak_infected = (T == 0) ? 0 : h[6];
            r.peak_step = (T == 0) ? 0u : (uint32_t)h[7];
            if (s0 != 0) {
                r.curve_mean = (double)s1 / (double)s0;
                const u128 a = s0 * s2, b = s1 * s1;
                r.curve_var = (double)(a - b) / ((double)s0 * (double)s0);
            }
            if (T) {
                int64_t last[4];
                AMB_TRY(copy_out(pop->series + (size_t)(T - 1) * 4u, last, sizeof(last), 0, s));
                r.final_s = last[0];
                r.final_i = last[1];
                r.final_r = last[2];
            }
        }
    }
    if (hist_len) *hist_len = bins_out;
    *out = r;
    return AMB_OK;
}

}  // extern "C"

namespace {
// One warp waits in the library's look-back for a predecessor tile that never
// publishes (its status word stays zero).
__global__ void wait_selfcheck_kernel(uint64_t *status, uint32_t *err, unsigned long long *ns)
{
    const uint64_t t0 = global_ns();
    (void)warp_lookback(status, 1u, 1u, 1u, err);
    if (threadIdx.x == 0) *ns = global_ns() - t0;
}
}  // namespace

extern "C" {

amb_status amb_debug_fail_creates(uint32_t k)
{
    g_fail_creates.store(k);
    return AMB_OK;
}

amb_status amb_selfcheck_wait_timeout(void *cuda_stream, double *waited_s)
{
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint64_t *status = nullptr;
    uint32_t *err = nullptr;
    unsigned long long *ns = nullptr;
    amb_status st = dalloc(&status, 2, s);
    if (st == AMB_OK) st = dalloc(&err, 1, s);
    if (st == AMB_OK) st = dalloc(&ns, 1, s);
    if (st == AMB_OK && (cudaMemsetAsync(status, 0, 2 * sizeof(uint64_t), s) != cudaSuccess ||
                         cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess))
        st = fail(AMB_ECUDA, "memset failed");
    uint32_t h_err = 0;
    unsigned long long h_ns = 0;
    if (st == AMB_OK) {
        wait_selfcheck_kernel<<<1, 32, 0, s>>>(status, err, ns);
        if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&h_ns, ns, sizeof(h_ns), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(AMB_ECUDA, "self-check kernel failed");
    }
    dfree(status, s);
    dfree(err, s);
    dfree(ns, s);
    cudaStreamSynchronize(s);
    AMB_TRY(st);
    if (waited_s) *waited_s = (double)h_ns * 1e-9;
    if (h_err & ERR_TIMEOUT) return fail(AMB_ETIMEOUT, "the wait gave up after %.3f s as designed", (double)h_ns * 1e-9);
    return fail(AMB_EINVARIANT, "the wait ended without its predecessor and without a timeout");
}

amb_status amb_cell_index(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *start, int32_t *ids,
                          void *cuda_stream, int sync)
{
    AMB_TRACE("amb_cell_index");
    if ((!x || !y || !ids) && n) return fail(AMB_EINVAL, "null pointer");
    if (!start) return fail(AMB_EINVAL, "null pointer");
    if (L < 1 || (uint64_t)L * L >= 0x80000000ull) return fail(AMB_EINVAL, "need 1 <= L and L*L < 2^31");
    if (n > 0x7FFFFFFFu) return fail(AMB_EINVAL, "n must be < 2^31");
    if (((uintptr_t)start & 15u) != 0) return fail(AMB_EINVAL, "start must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const uint64_t C = (uint64_t)L * L;
    int32_t *cnt = nullptr, *cursor = nullptr;
    uint32_t *err = nullptr;
    Lookback lb;
    amb_status st = dalloc(&cnt, C, s);
    if (st == AMB_OK) st = dalloc(&cursor, C, s);
    if (st == AMB_OK) st = dalloc(&err, 1, s);
    if (st == AMB_OK && cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess) st = fail(AMB_ECUDA, "memset");
    if (st == AMB_OK) st = launch_cell_index(x, y, n, L, start, ids, cnt, cursor, lb, err, s);
    uint32_t h = 0;
    if (st == AMB_OK && sync) {
        if (cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = fail(AMB_ECUDA, "sync failed");
    }
    dfree(cnt, s);
    dfree(cursor, s);
    dfree(err, s);
    lb.release(s);
    if (sync && cudaStreamSynchronize(s) != cudaSuccess && st == AMB_OK) st = fail(AMB_ECUDA, "sync failed");
    if (st == AMB_OK && (h & ERR_RANGE)) st = fail(AMB_EINVAL, "some coordinates were outside [0, L)");
    if (st == AMB_OK && (h & ERR_TIMEOUT)) st = fail(AMB_ETIMEOUT, "look-back wait ran out");
    return st;
}

}  // extern "C"
