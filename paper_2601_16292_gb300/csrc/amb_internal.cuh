// amb_internal.cuh -- population object and kernel launchers shared by the
// library's translation units (not part of the ABI).
#pragma once

#include <vector>

#include "amb_common.cuh"

#include <nvtx3/nvToolsExt.h>

namespace amb {

// NVTX range over one library call (header-only NVTX v3: a no-op unless a
// profiler such as Nsight Compute or Systems is attached).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
#define AMB_TRACE(name) ::amb::TraceRange amb_trace_range_(name)


// The library's stream-ordered memory pool on the current device: freed
// blocks stay cached in the pool (release threshold: never), so repeated
// allocations of view buffers, staging buffers and batch tables do not map
// and unmap device memory each time.  Falls back to the device's default
// pool if a pool cannot be created.
cudaMemPool_t library_pool();

// Stream-ordered device allocation helpers; every buffer of a population is
// allocated and freed on the population's stream.
template <class T>
amb_status dalloc(T **p, size_t count, cudaStream_t s)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaMemPool_t pool = library_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync((void **)p, count * sizeof(T), pool, s)
                         : cudaMallocAsync((void **)p, count * sizeof(T), s);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? AMB_ENOMEM : AMB_ECUDA,
                    "cudaMallocAsync(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
    }
    return AMB_OK;
}

template <class T>
void dfree(T *&p, cudaStream_t s)
{
    if (p) cudaFreeAsync((void *)p, s);
    p = nullptr;
}

// Look-back machinery shared by every single-pass scan launch of one owner:
// tile status words (epoch tagged, never cleared) and two ticket counters
// used alternately (each launch zeroes the counter of the next one).
struct Lookback {
    uint64_t *status = nullptr;
    size_t cap = 0;
    unsigned long long *tickets = nullptr;  // [2]
    uint32_t launches = 0;

    amb_status ensure(size_t tiles, cudaStream_t s);
    void release(cudaStream_t s);
    // parity and epoch of the next launch
    void next(uint32_t *parity, uint32_t *epoch)
    {
        *parity = launches & 1u;
        *epoch = (launches % 0x3FFFFFFFu) + 1u;
        ++launches;
    }
};

// Scan + scatter of the counting sort; scratch is owned by the caller.
struct CellIndexScratch {
    int32_t *cnt = nullptr;     // C
    int32_t *cursor = nullptr;  // C
    Lookback lb;
};

// Counting-sort cell index: start[C+1], ids[n] from id-ordered x, y.
// `cnt` must hold C int32; `cursor` C int32.  err gets ERR_RANGE for agents
// outside the grid (they are left out).
amb_status launch_cell_index(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *start,
                             int32_t *ids, int32_t *cnt, int32_t *cursor, Lookback &lb, uint32_t *err,
                             cudaStream_t s);
// The same index with every scratch buffer supplied by the caller (allocates
// nothing): cnt and cursor hold C int32, status scan_tiles(C) words, tickets
// two counters whose `parity` one is zero; epoch and parity advance per call
// as Lookback::next does.
uint32_t scan_tiles(uint32_t m);
amb_status launch_cell_index_raw(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *start,
                                 int32_t *ids, int32_t *cnt, int32_t *cursor, uint64_t *status,
                                 unsigned long long *tickets, uint32_t parity, uint32_t epoch, uint32_t *err,
                                 cudaStream_t s);
// ids[cursor[c]++] = i for every agent i in range (cursor = copy of start).
amb_status launch_cell_scatter(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L, int32_t *cursor,
                               int32_t *ids, cudaStream_t s);
// ---- batches: many populations advanced by one persistent launch ----
bool wealth_uses_smem(uint32_t n);
// Band shape of the SIR populations of a batch: rows per band at most
// rows_cap; spread = as many bands as fill the GPU, else the fewest bands.
struct BandShape {
    uint32_t rows_cap = 32;
    bool spread = false;
    // adaptive: spread when the fewest bands of all live populations would
    // not give every SM two bands, else fewest
    bool adaptive = false;
    // bytes of shared-memory counters a band may use (0: the single-population
    // kernel's budget)
    uint32_t smem_cap = 0;
};
// Re-derive a SIR population's band geometry for `shape` (records unchanged).
amb_status sir_band_regeometry(amb_pop *pop, BandShape shape);
// Fewest-bands count of an L x L grid under rows_cap (0 when unsupported).
uint32_t sir_fewest_bands(uint32_t L, uint32_t rows_cap, uint32_t smem_cap);

amb_status check_params(amb_model model, const amb_params *p, uint64_t seed);
bool injected_create_failure();

// Advance pops[i] by ks[i] steps with the batched launches (optionally as one
// CUDA graph); *launches += kernels launched, *ms = device time.
amb_status advance(const std::vector<amb_pop *> &pops, const std::vector<uint32_t> &ks, BandShape shape,
                   cudaStream_t s, bool graph, uint64_t *launches, float *ms);
// Device error words of the populations (one synchronisation), and the first
// one as a status.
amb_status read_errors(const std::vector<amb_pop *> &pops, cudaStream_t s, std::vector<uint32_t> &words);
amb_status check_errors(const std::vector<amb_pop *> &pops, cudaStream_t s);

// Step-count rows of a population: capacity for `rows` steps.
amb_status ensure_series(amb_pop *pop, uint64_t rows);

// Exclusive scan in[0..m) -> out[0..m], out[m] = total; out2 (optional) gets
// the same exclusive values.
amb_status launch_scan(const int32_t *in, int32_t *out, int32_t *out2, uint32_t m, Lookback &lb, uint32_t *err,
                       cudaStream_t s);

}  // namespace amb

// Band path record layout (SIR, cell-ordered records): one uint32 "aux" per
// record next to the agent id:
//   [15:0]  column after the next move (L <= 65536; the current column is
//           the cell's, found through start[])
//   [17:16] state                   [19:18] unused
//   [21:20] next move dy + 1
//   [22]    next-step recovery draw passed (infected agents)
//   [30:23] top byte of the next-step infection draw u1 (susceptible agents)
//   [31]    always 0
namespace amb {
constexpr uint32_t kAuxXMask = 0xFFFFu;
constexpr int kAuxStateShift = 16;
constexpr int kAuxDxShift = 18;
constexpr int kAuxDyShift = 20;
constexpr int kAuxRecShift = 22;
constexpr int kAuxCodeShift = 23;
}  // namespace amb

struct amb_pop {
    amb_model model;
    amb_params p;
    amb_cparams cp{};  // continuous-space models
    uint32_t key0 = 0, key1 = 0;
    cudaStream_t stream = nullptr;
    uint64_t t = 0;          // steps completed
    uint64_t launches = 0;   // kernels launched by step calls
    uint32_t path = 0;       // SIR: AMB_SIR_GENERIC or AMB_SIR_BAND

    // wealth
    int32_t *w = nullptr;
    int32_t *credit = nullptr;     // n, zero between steps (global path)
    int64_t ref_total = 0;         // total wealth the conservation check expects
    bool ref_total_valid = false;
    uint64_t conservation_from = 0;  // first step row the conservation check covers
    uint64_t monotone_from = 0;      // first step row the SIR count checks cover

    // walk / generic SIR: id-ordered columns
    int32_t *x = nullptr, *y = nullptr;
    uint8_t *state = nullptr;
    // SIR generic scratch
    int32_t *cnt = nullptr, *inf = nullptr, *cursor = nullptr;
    // cell index (SIR: rebuilt every step; walk: on demand)
    int32_t *start = nullptr, *ids = nullptr;
    bool index_valid = false;

    // SIR band path: cell-ordered records, double-buffered
    uint2 *rec[2] = {nullptr, nullptr};  // {id, word} per slot
    int32_t *row_start[2] = {nullptr, nullptr};
    int cur = 0;
    bool band_dirty = false;  // x, y, state hold written columns; records rebuilt before use
    uint32_t band_rows = 0, n_bands = 0;
    uint32_t band_grid = 0;
    uint32_t *band_wide = nullptr;  // per-CTA 32-bit counters in global memory (bands too dense for shared ones)
    bool band_narrow = false;       // 16-bit shared counters (bands twice as tall)
    uint32_t band_smem = 0;         // dynamic shared memory of the step kernel (bytes)

    // SIR thresholds
    uint32_t *t_inf_d = nullptr;
    std::vector<uint32_t> t_inf_h;
    uint32_t K = 0, t_rec = 0;
    int64_t init_infected = -1;

    // per-step counts: rows of 4 int64
    int64_t *series = nullptr;
    // amb_counts_async copies run on a side stream after an event recorded on
    // `stream`, so later steps do not wait for them; `stream` waits for
    // ev_copied before anything that synchronises the population or frees
    // `series`
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_ready = nullptr, ev_copied = nullptr;
    bool copies_pending = false;
    size_t series_cap = 0;
    bool series_next_zero = false;  // count row t is known to be zero (the last band step cleared it)

    // continuous-space models: float positions, days infected, and the
    // infected agents' positions in cell order (grid of cells wider than r)
    float *fx = nullptr, *fy = nullptr;
    int32_t *days = nullptr;
    int32_t *cell = nullptr;
    float2 *inf_pos = nullptr;

    amb::Lookback lb;
    uint32_t *err = nullptr;  // device error word (sticky)
};

namespace amb {
amb_status band_sync_records(amb_pop *pop);
bool is_continuous(const amb_pop *pop);
amb_status cont_steps(amb_pop *pop, uint32_t k);
amb_status cont_read_column(amb_pop *pop, amb_col col, void *dst, size_t n, int dst_on_device);
amb_status cont_write_column(amb_pop *pop, amb_col col, const void *src, size_t n, int src_on_device);
amb_status cont_bounds(amb_pop *pop, bool *ok);
void cont_release(amb_pop *pop);
}  // namespace amb
