// sir_band.cu -- SIR step over cell-ordered records, one fused kernel per step.
//
// Layout.  Agents are kept as records sorted by cell (c = y*L + x): rec_id[s]
// (agent id) and rec_aux[s] (x, state and the agent's draws for the next
// step, bit layout in amb_internal.cuh).  row_start[r] is the first slot of
// grid row r (row_start[L] = n); start[C+1] is the counting-sort cell index
// (grid environment, paper Sec. 4.1).  y is implied by the row a record sits
// in, so a record is 8 bytes.
//
// One step (synchronous semantics, paper Sec. 3.4).  A CTA owns a band of H
// grid rows.  A Moore move changes y by at most one, so every agent that lands
// in the band sits, before the move, in rows r0-1 .. r1 (torus wrap).  The CTA
//   1. reads those records and counts, in shared memory, agents and
//      start-of-step infected agents per new cell of the band (the cell
//      histogram and the per-cell infected counts k);
//   2. scans the band's counts (block-level exclusive scan) and gets the
//      band's first output slot from its predecessors by decoupled look-back
//      (bands are handed out in order by an atomic ticket);
//   3. writes start[] for its cells and row_start for its rows;
//   4. reads the records again and, for each agent landing in the band,
//      applies infection (k >= the agent's precomputed code) or recovery,
//      draws the agent's next-step Philox words (direction, infection code,
//      recovery bit) and scatters the record to its new slot.
// Per-step S / I / R / new-infection counts are warp-aggregated.
#include <algorithm>

#include "amb_internal.cuh"

namespace amb {

constexpr int kBandNT = 1024;
constexpr uint32_t kBandMaxCells = 24576;  // two uint32 counters per cell: 192 KiB
constexpr int kMaxSrcRows = 256;

struct BandArgs {
    const uint32_t *id_in;
    const uint32_t *aux_in;
    const int32_t *row_in;
    uint32_t *id_out;
    uint32_t *aux_out;
    int32_t *row_out;
    int32_t *start;
    uint32_t n, L, H, n_bands;
    uint32_t k0, k1, t;  // t = the step executed by this launch
    const uint32_t *t_inf;
    uint32_t K, t_rec;
    int64_t *row;  // the step's count row
    unsigned long long *tickets;
    uint32_t parity;
    uint64_t *status;
    uint32_t epoch;
    uint32_t *err;
};

// T_inf[min(k, K)] for k = 0 .. 254, and T_inf[K].
__device__ __forceinline__ void load_tinf(uint32_t *tinf_s, const uint32_t *t_inf, uint32_t K)
{
    for (uint32_t i = threadIdx.x; i <= kCodeTable; i += blockDim.x) tinf_s[i] = t_inf[i < K ? i : K];
}

// Next-step draw bits of one agent: direction (u0 >> 29), recovery bit
// (u2 < T_rec) and the infection code of u1: the smallest k in [1, K] with
// u1 < T_inf[k] when it is <= 254, 255 when it is larger, 0 when none.
__device__ __forceinline__ uint32_t draw_bits(uint32_t id, uint32_t t, uint32_t k0, uint32_t k1,
                                              const uint32_t *tinf_s, uint32_t K, uint32_t tinf_max, uint32_t t_rec)
{
    const U4 u = philox(id, t, k0, k1);
    const uint32_t dir = u.w0 >> 29;
    const uint32_t rec = (u.w2 < t_rec) ? 1u : 0u;
    const uint32_t u1 = u.w1;
    uint32_t k = 0;  // largest k in [0, 254] with T_inf[min(k,K)] <= u1
#pragma unroll
    for (uint32_t step = 128; step >= 1; step >>= 1)
        if (k + step <= kCodeTable && tinf_s[k + step] <= u1) k += step;
    uint32_t code;
    if (k < kCodeTable)
        code = k + 1;
    else
        code = (K > kCodeTable && u1 < tinf_max) ? kCodeExact : 0u;
    return (dir << kAuxDirShift) | (rec << kAuxRecShift) | (code << kAuxCodeShift);
}

__device__ __forceinline__ uint32_t find_src_row(const uint32_t *srow, uint32_t nsrc, uint32_t v)
{
    uint32_t lo = 0, hi = nsrc - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (srow[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kBandNT, 1) sir_band_kernel(const BandArgs a)
{
    extern __shared__ __align__(16) uint32_t band_smem[];
    __shared__ uint32_t tinf_s[kCodeTable + 2];
    __shared__ uint32_t srow[kMaxSrcRows + 1];
    __shared__ uint32_t sbase[kMaxSrcRows];
    __shared__ uint32_t sy[kMaxSrcRows];
    __shared__ uint32_t s_warp[kBandNT / 32 + 1];
    __shared__ uint32_t s_band, s_prefix, s_nsrc;
    __shared__ unsigned long long s_cnt[4];

    const uint32_t L = a.L, H = a.H;
    uint32_t *cnt = band_smem;          // H*L: agents per new cell, then slot cursors
    uint32_t *inf = band_smem + H * L;  // H*L: start-of-step infected per new cell
    const uint32_t tid = threadIdx.x;

    if (blockIdx.x == 0 && tid == 0) a.tickets[a.parity ^ 1u] = 0ull;
    load_tinf(tinf_s, a.t_inf, a.K);
    if (tid < 4) s_cnt[tid] = 0ull;
    const uint32_t tinf_max = a.t_inf[a.K];
    const uint32_t t_next = a.t + 1u;
    uint32_t cS = 0, cI = 0, cR = 0, cNew = 0;
    const bool single = (a.n_bands == 1);

    for (;;) {
        if (tid == 0) s_band = (uint32_t)atomicAdd(&a.tickets[a.parity], 1ull);
        __syncthreads();
        const uint32_t b = s_band;
        if (b >= a.n_bands) break;
        const uint32_t r0 = b * H;
        const uint32_t r1 = min(r0 + H, L);
        const uint32_t rows = r1 - r0;
        const uint32_t cells = rows * L;
        for (uint32_t i = tid; i < cells; i += kBandNT) {
            cnt[i] = 0u;
            inf[i] = 0u;
        }
        if (tid == 0) {
            const uint32_t nsrc = single ? L : rows + 2u;
            uint32_t v = 0;
            for (uint32_t j = 0; j < nsrc; ++j) {
                const uint32_t y = single ? j : (r0 + L - 1u + j) % L;
                const int32_t beg = a.row_in[y], end = a.row_in[y + 1];
                srow[j] = v;
                sbase[j] = (uint32_t)beg;
                sy[j] = y;
                v += (uint32_t)(end - beg);
            }
            srow[nsrc] = v;
            s_nsrc = nsrc;
        }
        __syncthreads();
        const uint32_t nsrc = s_nsrc;
        const uint32_t M = srow[nsrc];

        // pass 1: histogram of new cells and start-of-step infected per new cell
        for (uint32_t v = tid; v < M; v += kBandNT) {
            const uint32_t j = find_src_row(srow, nsrc, v);
            const uint32_t s = sbase[j] + (v - srow[j]);
            if (s >= a.n) {
                atomicOr(a.err, ERR_RANGE);
                continue;
            }
            const uint32_t aux = a.aux_in[s];
            const uint32_t x = aux & kAuxXMask;
            if (x >= L) {
                atomicOr(a.err, ERR_RANGE);
                continue;
            }
            const uint32_t d = (aux >> kAuxDirShift) & 7u;
            const uint32_t yn = (uint32_t)ring_add((int32_t)sy[j], dir_dy(d), (int32_t)L);
            if (yn < r0 || yn >= r1) continue;
            const uint32_t xn = (uint32_t)ring_add((int32_t)x, dir_dx(d), (int32_t)L);
            const uint32_t c = (yn - r0) * L + xn;
            atomicAdd(&cnt[c], 1u);
            if (((aux >> kAuxStateShift) & 3u) == AMB_I) atomicAdd(&inf[c], 1u);
        }
        __syncthreads();

        // exclusive scan of the band's cell counts, in place
        uint32_t running = 0;
        for (uint32_t base = 0; base < cells; base += kBandNT * 4u) {
            const uint32_t i0 = base + tid * 4u;
            uint32_t q[4];
            if (i0 + 3u < cells) {
                const uint4 w = *reinterpret_cast<const uint4 *>(&cnt[i0]);
                q[0] = w.x; q[1] = w.y; q[2] = w.z; q[3] = w.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) q[e] = (i0 + e < cells) ? cnt[i0 + e] : 0u;
            }
            uint32_t total;
            const uint32_t ex = block_exclusive_scan<kBandNT>(q[0] + q[1] + q[2] + q[3], s_warp, &total);
            uint32_t e0 = running + ex;
            uint32_t o[4];
            o[0] = e0; o[1] = o[0] + q[0]; o[2] = o[1] + q[1]; o[3] = o[2] + q[2];
            if (i0 + 3u < cells) {
                *reinterpret_cast<uint4 *>(&cnt[i0]) = make_uint4(o[0], o[1], o[2], o[3]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i0 + e < cells) cnt[i0 + e] = o[e];
            }
            running += total;
        }
        // first output slot of the band
        if (tid == 0) s_prefix = lookback_exclusive(a.status, b, a.epoch, running, a.err);
        __syncthreads();
        const uint32_t P = s_prefix;
        const uint32_t T = running;

        // cell index and row starts of the band
        int32_t *start_band = a.start + (size_t)r0 * L;
        for (uint32_t i = tid; i < cells; i += kBandNT) start_band[i] = (int32_t)(P + cnt[i]);
        for (uint32_t r = tid; r < rows; r += kBandNT) a.row_out[r0 + r] = (int32_t)(P + cnt[r * L]);
        if (b == a.n_bands - 1u && tid == 0) {
            a.start[(size_t)L * L] = (int32_t)(P + T);
            a.row_out[L] = (int32_t)(P + T);
        }
        __syncthreads();

        // pass 2: transitions, next draws, scatter
        for (uint32_t v = tid; v < M; v += kBandNT) {
            const uint32_t j = find_src_row(srow, nsrc, v);
            const uint32_t s = sbase[j] + (v - srow[j]);
            if (s >= a.n) continue;
            const uint32_t aux = a.aux_in[s];
            const uint32_t x = aux & kAuxXMask;
            if (x >= L) continue;
            const uint32_t d = (aux >> kAuxDirShift) & 7u;
            const uint32_t yn = (uint32_t)ring_add((int32_t)sy[j], dir_dy(d), (int32_t)L);
            if (yn < r0 || yn >= r1) continue;
            const uint32_t xn = (uint32_t)ring_add((int32_t)x, dir_dx(d), (int32_t)L);
            const uint32_t c = (yn - r0) * L + xn;
            const uint32_t id = a.id_in[s];
            uint32_t st = (aux >> kAuxStateShift) & 3u;
            if (st == AMB_S) {
                const uint32_t code = aux >> kAuxCodeShift;
                const uint32_t k = inf[c];
                if (code != 0u && k >= code) {
                    bool hit = true;
                    if (code == kCodeExact) {
                        const U4 u = philox(id, a.t, a.k0, a.k1);
                        hit = u.w1 < a.t_inf[k < a.K ? k : a.K];
                    }
                    if (hit) {
                        st = AMB_I;
                        ++cNew;
                    }
                }
            } else if (st == AMB_I) {
                if ((aux >> kAuxRecShift) & 1u) st = AMB_R;
            }
            cS += (st == AMB_S);
            cI += (st == AMB_I);
            cR += (st == AMB_R);
            const uint32_t slot = P + atomicAdd(&cnt[c], 1u);
            if (slot >= a.n) {
                atomicOr(a.err, ERR_OVERFLOW);
                continue;
            }
            const uint32_t naux =
                xn | (st << kAuxStateShift) | draw_bits(id, t_next, a.k0, a.k1, tinf_s, a.K, tinf_max, a.t_rec);
            a.id_out[slot] = id;
            a.aux_out[slot] = naux;
        }
        __syncthreads();
    }

    // per-step counts
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cS += __shfl_down_sync(0xffffffffu, cS, o);
        cI += __shfl_down_sync(0xffffffffu, cI, o);
        cR += __shfl_down_sync(0xffffffffu, cR, o);
        cNew += __shfl_down_sync(0xffffffffu, cNew, o);
    }
    if ((tid & 31u) == 0) {
        if (cS) atomicAdd(&s_cnt[0], (unsigned long long)cS);
        if (cI) atomicAdd(&s_cnt[1], (unsigned long long)cI);
        if (cR) atomicAdd(&s_cnt[2], (unsigned long long)cR);
        if (cNew) atomicAdd(&s_cnt[3], (unsigned long long)cNew);
    }
    __syncthreads();
    if (tid < 4 && s_cnt[tid]) atomicAdd(reinterpret_cast<unsigned long long *>(&a.row[tid]), s_cnt[tid]);
}

// ------------------------------------------------------------- set-up ---
// Records of the agents from id-ordered columns: ids already in cell order.
__global__ void band_build_kernel(const uint32_t *__restrict__ ids, const int32_t *__restrict__ x,
                                  const uint8_t *__restrict__ state, uint32_t n, uint32_t *__restrict__ aux,
                                  uint32_t k0, uint32_t k1, uint32_t t, const uint32_t *__restrict__ t_inf,
                                  uint32_t K, uint32_t t_rec)
{
    __shared__ uint32_t tinf_s[kCodeTable + 2];
    load_tinf(tinf_s, t_inf, K);
    __syncthreads();
    const uint32_t tinf_max = t_inf[K];
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t id = ids[s];
        if (id >= n) continue;  // only slots of agents left out of the index
        aux[s] = (uint32_t)x[id] | ((uint32_t)state[id] << kAuxStateShift) |
                 draw_bits(id, t, k0, k1, tinf_s, K, tinf_max, t_rec);
    }
}

__global__ void band_rows_kernel(const int32_t *__restrict__ start, uint32_t L, int32_t *__restrict__ row_start)
{
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r <= L; r += gridDim.x * blockDim.x)
        row_start[r] = start[(size_t)r * L];
}

// id-ordered column from the records
__global__ void band_read_kernel(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ aux,
                                 const int32_t *__restrict__ row_start, uint32_t n, uint32_t L, int col,
                                 void *__restrict__ out)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t id = ids[s];
        if (id >= n) continue;
        const uint32_t a = aux[s];
        if (col == AMB_COL_X) {
            static_cast<int32_t *>(out)[id] = (int32_t)(a & kAuxXMask);
        } else if (col == AMB_COL_STATE) {
            static_cast<uint8_t *>(out)[id] = (uint8_t)((a >> kAuxStateShift) & 3u);
        } else {
            uint32_t lo = 0, hi = L - 1;  // largest row r with row_start[r] <= s
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if ((uint32_t)row_start[mid] <= s)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            static_cast<int32_t *>(out)[id] = (int32_t)lo;
        }
    }
}

static int sm_count()
{
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

bool sir_band_supported(uint32_t L, uint32_t *band_rows)
{
    *band_rows = 0;
    if (L < 1 || L > 0xFFFFu || L > kBandMaxCells) return false;
    if ((uint64_t)L * L <= kBandMaxCells) {
        *band_rows = L;  // one band holds the whole grid
        return true;
    }
    const uint32_t by_smem = kBandMaxCells / L;
    const uint32_t target = std::max<uint32_t>(1u, (L + 2u * 152u - 1u) / (2u * 152u));
    uint32_t H = std::min<uint32_t>(by_smem, std::max<uint32_t>(1u, target));
    H = std::min<uint32_t>(H, L - 2u);
    *band_rows = std::max<uint32_t>(H, 1u);
    return true;
}

amb_status sir_band_init(amb_pop *pop, const int32_t *x, const int32_t *y, const uint8_t *state)
{
    cudaStream_t s = pop->stream;
    const uint32_t n = pop->p.n, L = pop->p.grid_side;
    const uint64_t C = (uint64_t)L * L;
    uint32_t H = 0;
    if (!sir_band_supported(L, &H)) return fail(AMB_EINVAL, "band path does not support L = %u", L);
    pop->band_rows = H;
    pop->n_bands = (L + H - 1) / H;
    for (int b = 0; b < 2; ++b) {
        if (!pop->rec_id[b]) AMB_TRY(dalloc(&pop->rec_id[b], n, s));
        if (!pop->rec_aux[b]) AMB_TRY(dalloc(&pop->rec_aux[b], n, s));
        if (!pop->row_start[b]) AMB_TRY(dalloc(&pop->row_start[b], (size_t)L + 1, s));
    }
    if (!pop->start) AMB_TRY(dalloc(&pop->start, C + 1, s));
    int32_t *cnt = nullptr, *cursor = nullptr;
    AMB_TRY(dalloc(&cnt, C, s));
    AMB_TRY(dalloc(&cursor, C, s));
    // agents into cell order; the id list becomes rec_id of the new buffer
    const int nb = pop->cur ^ 1;
    amb_status st = launch_cell_index(x, y, n, L, pop->start, (int32_t *)pop->rec_id[nb], cnt, cursor, pop->lb,
                                      pop->err, s);
    dfree(cnt, s);
    dfree(cursor, s);
    AMB_TRY(st);
    if (n) {
        band_build_kernel<<<grid_for(n, 256, 152u * 8u), 256, 0, s>>>(pop->rec_id[nb], x, state, n, pop->rec_aux[nb],
                                                                       pop->key0, pop->key1, (uint32_t)pop->t,
                                                                       pop->t_inf_d, pop->K, pop->t_rec);
        AMB_TRY_CUDA(cudaGetLastError());
    }
    band_rows_kernel<<<grid_for((uint64_t)L + 1, 256), 256, 0, s>>>(pop->start, L, pop->row_start[nb]);
    AMB_TRY_CUDA(cudaGetLastError());
    pop->cur = nb;
    AMB_TRY(pop->lb.ensure(pop->n_bands, s));
    return AMB_OK;
}

amb_status sir_band_steps(amb_pop *pop, uint32_t k)
{
    cudaStream_t s = pop->stream;
    int64_t *rows = pop->series + (size_t)pop->t * 4u;
    AMB_TRY_CUDA(cudaMemsetAsync(rows, 0, (size_t)k * 4u * sizeof(int64_t), s));
    if (pop->p.n == 0) return AMB_OK;
    const uint32_t L = pop->p.grid_side, H = pop->band_rows;
    const size_t smem = (size_t)2u * H * L * sizeof(uint32_t);
    AMB_TRY_CUDA(cudaFuncSetAttribute(sir_band_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = std::min<unsigned>(pop->n_bands, (unsigned)sm_count());
    AMB_TRY(pop->lb.ensure(pop->n_bands, s));
    for (uint32_t j = 0; j < k; ++j) {
        BandArgs a;
        const int in = pop->cur, out = pop->cur ^ 1;
        a.id_in = pop->rec_id[in];
        a.aux_in = pop->rec_aux[in];
        a.row_in = pop->row_start[in];
        a.id_out = pop->rec_id[out];
        a.aux_out = pop->rec_aux[out];
        a.row_out = pop->row_start[out];
        a.start = pop->start;
        a.n = pop->p.n;
        a.L = L;
        a.H = H;
        a.n_bands = pop->n_bands;
        a.k0 = pop->key0;
        a.k1 = pop->key1;
        a.t = (uint32_t)(pop->t + j);
        a.t_inf = pop->t_inf_d;
        a.K = pop->K;
        a.t_rec = pop->t_rec;
        a.row = rows + (size_t)j * 4u;
        a.tickets = pop->lb.tickets;
        a.status = pop->lb.status;
        pop->lb.next(&a.parity, &a.epoch);
        a.err = pop->err;
        sir_band_kernel<<<grid, kBandNT, smem, s>>>(a);
        AMB_TRY_CUDA(cudaGetLastError());
        pop->cur = out;
        pop->launches += 1;
    }
    return AMB_OK;
}

amb_status sir_band_read(amb_pop *pop, amb_col col, void *dst_dev)
{
    const uint32_t n = pop->p.n;
    if (n == 0) return AMB_OK;
    band_read_kernel<<<grid_for(n, 256, 152u * 8u), 256, 0, pop->stream>>>(
        pop->rec_id[pop->cur], pop->rec_aux[pop->cur], pop->row_start[pop->cur], n, pop->p.grid_side, (int)col, dst_dev);
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
        dfree(pop->rec_id[b], pop->stream);
        dfree(pop->rec_aux[b], pop->stream);
        dfree(pop->row_start[b], pop->stream);
    }
}

}  // namespace amb
