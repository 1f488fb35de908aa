// sir_band.cu -- the SIR step of one population over cell-ordered records,
// one fused kernel launch per step (the band code is in band_device.cuh):
// step launches, set-up of the records from id-ordered columns, read-back of
// columns and of the cell index, and the band geometry of a grid.
#include <algorithm>
#include <cstring>

#include "band_device.cuh"

namespace amb {

// kNarrow: 16-bit shared counters (bands twice as tall), else 32-bit ones
template <bool kNarrow>
__global__ void __launch_bounds__(kBandNT, kBandCtasPerSm) sir_band_kernel(const BandArgs a)
{
    extern __shared__ __align__(16) uint32_t band_smem[];
    __shared__ BandShared sh;
    const uint32_t tid = threadIdx.x;

    // Bands are handed out in increasing order by ticket.  A CTA draws the
    // ticket of its next band during the current band's pass 2; the smallest
    // unfinished band is always some CTA's current one (all CTAs are
    // resident), so every look-back ends.  The first ticket is drawn before
    // the threshold table is loaded, so that its latency overlaps the loads.
    unsigned long long ticket = 0;
    if (tid == 0) ticket = atomicAdd(&a.tickets[a.parity], 1ull);
    if (blockIdx.x == 0 && tid == 0) a.tickets[a.parity ^ 1u] = 0ull;
    // the next step's launch adds into its row only after this one ends
    if (blockIdx.x == 0 && tid < 4 && a.row_next) a.row_next[tid] = 0;
    if (tid < 4) sh.cnt[tid] = 0ull;
    for (uint32_t i = tid; i < 256u; i += kBandNT) sh.ct.tinf[i] = a.t_inf[i < a.K ? i : a.K];
    if (tid == 0) sh.band = (uint32_t)ticket;
    __syncthreads();
    Tally tl = {0u, 0u, 0u, 0u};
    uint32_t *wide_slice = a.wide ? a.wide + (size_t)blockIdx.x * 2u * a.H * a.L : nullptr;
    for (uint32_t b = sh.band; b < a.n_bands; b = sh.band)
        process_band<true, false, true, kNarrow>(a, sh, band_smem, wide_slice, b, tl);
    flush_tally(sh, tl, a.row);
}

// ------------------------------------------------------------- set-up ---
// Records of the agents from id-ordered columns: ids already in cell order.
struct BuildArgs {
    const int32_t *ids;
    const int32_t *x;
    const uint8_t *state;
    uint32_t n, L;
    uint2 *rec;
    uint32_t t;
    uint32_t rk0[10], rk1[10];
    uint32_t t_rec;
};

__global__ void band_build_kernel(const BuildArgs a)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += gridDim.x * blockDim.x) {
        const uint32_t id = (uint32_t)a.ids[s];
        if (id >= a.n) continue;  // only slots of agents left out of the index
        const uint32_t st = a.state[id];
        a.rec[s] = make_uint2(id, record_word(id, a.t, st, (uint32_t)a.x[id], a.L, a.rk0, a.rk1, a.t_rec));
    }
}

__global__ void band_rows_kernel(const int32_t *__restrict__ start, uint32_t L, int32_t *__restrict__ row_start)
{
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r <= L; r += gridDim.x * blockDim.x)
        row_start[r] = start[(size_t)r * L];
}

// id-ordered column from the records
__global__ void band_read_kernel(const uint2 *__restrict__ rec, const int32_t *__restrict__ row_start,
                                 const int32_t *__restrict__ start, uint32_t n, uint32_t L, int col,
                                 void *__restrict__ out)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint2 r = rec[s];
        const uint32_t id = r.x;
        if (id >= n) continue;
        if (col == AMB_COL_STATE) {
            static_cast<uint8_t *>(out)[id] = (uint8_t)((r.y >> kAuxStateShift) & 3u);
            continue;
        }
        if (col == -1) {  // the ids in cell order (the cell index's id list)
            static_cast<int32_t *>(out)[s] = (int32_t)id;
            continue;
        }
        uint32_t lo = 0, hi = L - 1;  // row: largest r with row_start[r] <= s
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if ((uint32_t)row_start[mid] <= s)
                lo = mid;
            else
                hi = mid - 1;
        }
        if (col == AMB_COL_Y) {
            static_cast<int32_t *>(out)[id] = (int32_t)lo;
            continue;
        }
        // column: largest x with start[y L + x] <= s (the record itself holds
        // the column after the agent's next move)
        const int32_t *row = start + (size_t)lo * L;
        uint32_t xl = 0, xh = L - 1;
        while (xl < xh) {
            const uint32_t mid = (xl + xh + 1) >> 1;
            if ((uint32_t)row[mid] <= s)
                xl = mid;
            else
                xh = mid - 1;
        }
        static_cast<int32_t *>(out)[id] = (int32_t)xl;
    }
}


// Band geometry for an L x L grid, grid_max CTAs:
//  * H (rows of the tallest band, <= 32) as large as the shared-memory
//    counters allow (one word per cell);
//  * n_bands a multiple of the grid (every CTA gets the same number of
//    bands; band b covers rows [b L / n_bands, (b+1) L / n_bands));
//  * one band when the whole grid fits (L <= 32).
struct BandGeometry {
    uint32_t H, n_bands, smem;
};

// Band geometry of an L x L grid: single band when the whole grid fits,
// else bands of at most min(rows_cap, smem, L - 2) rows (L - 2 keeps a band's
// rows + 2 source rows distinct).  spread: as many bands as fill grid_max CTAs
// (the whole GPU works on one population); otherwise the fewest bands (many
// populations share the GPU in a batch).
static bool band_geometry(uint32_t L, uint32_t grid_max, BandGeometry *g, uint32_t rows_cap = kMaxBandRows,
                          bool spread = true, uint32_t smem_cap = 0, bool narrow = false)
{
    // bytes of shared counters per cell: 4, or 2 with 16-bit counters
    const uint32_t cell_bytes = narrow ? 2u : 4u;
    // counters of at most `budget` bytes (kBandSmem, or less for a kernel
    // with more static shared memory); the round-up to groups of four words
    // adds at most 12 bytes, which the kernels' limits leave room for
    const uint32_t budget = smem_cap ? std::min<uint32_t>(smem_cap, kBandSmem) : kBandSmem;
    if (L < 1 || L > 0xFFFFu || (uint64_t)L * cell_bytes > budget) return false;
    if (narrow && (L % 8u != 0 || L > 8192u)) return false;
    rows_cap = std::max<uint32_t>(1u, std::min<uint32_t>(rows_cap, kMaxBandRows));
    const uint32_t by_smem = budget / (L * cell_bytes);
    uint32_t H, nb;
    if ((L <= rows_cap || L <= 2u) && L <= by_smem) {
        H = L;
        nb = 1;
    } else {
        const uint32_t h = std::max<uint32_t>(
            1u, std::min<uint32_t>(std::min<uint32_t>(rows_cap, by_smem), L > 2u ? L - 2u : 1u));
        if (spread) {
            const uint32_t waves = (L + grid_max * h - 1u) / (grid_max * h);
            nb = std::min<uint32_t>(L, grid_max * waves);
        } else {
            nb = (L + h - 1u) / h;
        }
        H = (L + nb - 1u) / nb;
    }
    g->H = H;
    g->n_bands = nb;
    g->smem = narrow ? ((H * L / 2u + 3u) & ~3u) * 4u : ((H * L + 3u) & ~3u) * 4u;
    return true;
}

// 16-bit counters for a population: always with AMB_SIR_BAND16, never with
// AMB_SIR_BAND32; otherwise when they need fewer waves of bands than 32-bit
// ones and rows hold at most 3,072 agents on average (a row must stay below
// 4,096; a band where one does not is redone with 32-bit counters).
static bool choose_narrow(const amb_pop *pop, uint32_t grid_max)
{
    const uint32_t L = pop->p.grid_side;
    BandGeometry g32, g16;
    if (pop->p.variant == AMB_SIR_BAND32 || !band_geometry(L, grid_max, &g16, kMaxBandRows, true, 0, true))
        return false;
    if (pop->p.variant == AMB_SIR_BAND16) return true;
    return band_geometry(L, grid_max, &g32) && g16.n_bands < g32.n_bands && (uint64_t)pop->p.n <= 3072ull * L;
}

uint32_t sir_fewest_bands(uint32_t L, uint32_t rows_cap, uint32_t smem_cap)
{
    BandGeometry g;
    return band_geometry(L, device_sms() * kBandCtasPerSm, &g, rows_cap, false, smem_cap) ? g.n_bands : 0u;
}

bool sir_band_supported(uint32_t L, uint32_t *band_rows)
{
    BandGeometry g;
    if (!band_geometry(L, device_sms() * kBandCtasPerSm, &g)) return false;
    *band_rows = g.H;
    return true;
}

amb_status sir_band_init(amb_pop *pop, const int32_t *x, const int32_t *y, const uint8_t *state)
{
    cudaStream_t s = pop->stream;
    const uint32_t n = pop->p.n, L = pop->p.grid_side;
    const uint64_t C = (uint64_t)L * L;
    const uint32_t grid_max = device_sms() * kBandCtasPerSm;
    BandGeometry g;
    const bool narrow = choose_narrow(pop, grid_max);
    if (!band_geometry(L, grid_max, &g, kMaxBandRows, true, 0, narrow))
        return fail(AMB_EINVAL, "band path does not support L = %u", L);
    const uint32_t H = g.H;
    pop->band_narrow = narrow;
    pop->band_rows = H;
    pop->n_bands = g.n_bands;
    pop->band_grid = std::min<uint32_t>(g.n_bands, grid_max);
    pop->band_smem = g.smem;
    for (int b = 0; b < 2; ++b) {
        // 4 spare entries past the last record (slack; no kernel reads them)
        if (!pop->rec[b]) AMB_TRY(dalloc(&pop->rec[b], (size_t)n + 4u, s));
        if (!pop->row_start[b]) AMB_TRY(dalloc(&pop->row_start[b], (size_t)L + 1, s));
    }
    if (!pop->start) AMB_TRY(dalloc(&pop->start, C + 1, s));
    int32_t *cnt = nullptr, *cursor = nullptr;
    AMB_TRY(dalloc(&cnt, C, s));
    AMB_TRY(dalloc(&cursor, C, s));
    // agents into cell order, then their records into the new buffer
    const int nb = pop->cur ^ 1;
    int32_t *ids = nullptr;
    amb_status st = dalloc(&ids, n, s);
    if (st == AMB_OK)
        st = launch_cell_index(x, y, n, L, pop->start, ids, cnt, cursor, pop->lb, pop->err, s);
    dfree(cnt, s);
    dfree(cursor, s);
    if (st != AMB_OK) {
        dfree(ids, s);
        return st;
    }
    if (n) {
        BuildArgs b;
        b.ids = ids;
        b.x = x;
        b.state = state;
        b.n = n;
        b.L = L;
        b.rec = pop->rec[nb];
        b.t = (uint32_t)pop->t;
        round_keys(pop->key0, pop->key1, b.rk0, b.rk1);
        b.t_rec = pop->t_rec;
        band_build_kernel<<<grid_for(n, 256, 8u), 256, 0, s>>>(b);
    }
    dfree(ids, s);
    AMB_TRY_CUDA(cudaGetLastError());
    band_rows_kernel<<<grid_for((uint64_t)L + 1, 256), 256, 0, s>>>(pop->start, L, pop->row_start[nb]);
    AMB_TRY_CUDA(cudaGetLastError());
    pop->cur = nb;
    AMB_TRY(pop->lb.ensure(pop->n_bands, s));
    return AMB_OK;
}

amb_status sir_band_steps(amb_pop *pop, uint32_t k)
{
    cudaStream_t s = pop->stream;
    // every launch clears the next step's count row, so only the first row
    // needs clearing here, and not even that after a band step of this
    // population (one more row of capacity keeps the last launch's next row)
    AMB_TRY(ensure_series(pop, pop->t + k + 1));
    int64_t *rows = pop->series + (size_t)pop->t * 4u;
    if (pop->p.n == 0) {
        AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)(k + 1) * 4u * sizeof(int64_t), s));
        pop->series_next_zero = true;
        return AMB_OK;
    }
    if (!pop->series_next_zero) AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, 4u * sizeof(int64_t), s));
    pop->series_next_zero = false;
    const size_t smem = pop->band_smem;
    void (*const kernel)(BandArgs) = pop->band_narrow ? sir_band_kernel<true> : sir_band_kernel<false>;
    AMB_TRY_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    AMB_TRY(pop->lb.ensure(pop->n_bands, s));
    // 32-bit per-CTA counters for bands whose source rows hold >= 65536 agents,
    // or that do not fit 16-bit counters (allocated on the first step that may
    // need them; batched steps use their own)
    if ((pop->p.n >= kPackedLimit || pop->band_narrow) && !pop->band_wide)
        AMB_TRY(dalloc(&pop->band_wide, (size_t)pop->band_grid * 2u * pop->band_rows * pop->p.grid_side, s));
    BandArgs a;
    round_keys(pop->key0, pop->key1, a.rk0, a.rk1);
    for (uint32_t j = 0; j < k; ++j) {
        const int in = pop->cur, out = pop->cur ^ 1;
        a.rec_in = pop->rec[in];
        a.row_in = pop->row_start[in];
        a.rec_out = pop->rec[out];
        a.row_out = pop->row_start[out];
        a.start = pop->start;
        a.wide = pop->band_wide;
        a.n = pop->p.n;
        a.L = pop->p.grid_side;
        a.H = pop->band_rows;
        a.n_bands = pop->n_bands;
        a.k0 = pop->key0;
        a.k1 = pop->key1;
        a.t = (uint32_t)(pop->t + j);
        a.t_inf = pop->t_inf_d;
        a.K = pop->K;
        a.t_rec = pop->t_rec;
        a.row = rows + (size_t)j * 4u;
        a.row_next = rows + (size_t)(j + 1) * 4u;
        a.tickets = pop->lb.tickets;
        a.status = pop->lb.status;
        pop->lb.next(&a.parity, &a.epoch);
        a.err = pop->err;
        a.code_tab = nullptr;
        kernel<<<pop->band_grid, kBandNT, smem, s>>>(a);
        AMB_TRY_CUDA(cudaGetLastError());
        pop->cur = out;
        pop->launches += 1;
    }
    pop->series_next_zero = true;
    return AMB_OK;
}

amb_status sir_band_read(amb_pop *pop, amb_col col, void *dst_dev)
{
    const uint32_t n = pop->p.n;
    if (n == 0) return AMB_OK;
    band_read_kernel<<<grid_for(n, 256, 8u), 256, 0, pop->stream>>>(
        pop->rec[pop->cur], pop->row_start[pop->cur], pop->start, n, pop->p.grid_side, (int)col, dst_dev);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status launch_occupancy_from_start(const int32_t *start, uint64_t C, int32_t *occ, cudaStream_t s);

amb_status sir_band_occupancy(amb_pop *pop, int32_t *occ)
{
    const uint64_t C = (uint64_t)pop->p.grid_side * pop->p.grid_side;
    return launch_occupancy_from_start(pop->start, C, occ, pop->stream);
}

void sir_band_release(amb_pop *pop)
{
    for (int b = 0; b < 2; ++b) {
        dfree(pop->rec[b], pop->stream);
        dfree(pop->row_start[b], pop->stream);
    }
    dfree(pop->band_wide, pop->stream);
}

}  // namespace amb

namespace amb {

// ------------------------------------------------------- batch, host side ---
// Re-derive the band geometry of a population with at most rows_cap rows per
// band (the records do not depend on it).
amb_status sir_band_regeometry(amb_pop *pop, BandShape shape)
{
    cudaStream_t s = pop->stream;
    const uint32_t L = pop->p.grid_side;
    const uint32_t grid_max = device_sms() * kBandCtasPerSm;
    BandGeometry g;
    if (!band_geometry(L, grid_max, &g, shape.rows_cap, shape.spread, shape.smem_cap))
        return fail(AMB_EINVAL, "band path does not support L = %u", L);
    const bool grow = (size_t)g.H * L > (size_t)pop->band_rows * L || std::min<uint32_t>(g.n_bands, grid_max) > pop->band_grid;
    pop->band_narrow = false;  // batches run 32-bit counters
    pop->band_rows = g.H;
    pop->n_bands = g.n_bands;
    pop->band_grid = std::min<uint32_t>(g.n_bands, grid_max);
    pop->band_smem = g.smem;
    if (pop->band_wide && grow) {  // re-sized on the next single-population step
        dfree(pop->band_wide, s);
        pop->band_wide = nullptr;
    }
    AMB_TRY(pop->lb.ensure(pop->n_bands, s));
    return AMB_OK;
}

}  // namespace amb
