// band_device.cuh -- device code of the SIR step over cell-ordered records:
// one band of grid rows per CTA, used by the single-population step kernel
// (sir_band.cu) and the persistent batch kernel (batch.cu).
//
// Layout.  Agents are kept as 8-byte records sorted by cell (c = y*L + x):
// rec[s] = {agent id, word}, the word holding x, state and the agent's draws
// for the next step (bit layout in amb_internal.cuh); id and word sit side by
// side so a record moves with one 64-bit load or store.  row_start[r] is the first slot of
// grid row r (row_start[L] = n); start[C+1] is the counting-sort cell index
// (grid environment, paper Sec. 4.1).  y is implied by the row a record sits
// in, so a record is 8 bytes.
//
// One step (synchronous semantics, paper Sec. 3.4).  A CTA owns a band of at
// most 32 grid rows.  A Moore move changes y by at most one, so every agent
// that lands in the band sits, before the move, in rows r0-1 .. r1 (torus
// wrap).  The CTA
//   1. reads those records and counts, in shared memory, agents and
//      start-of-step infected agents per new cell of the band (the cell
//      histogram and the per-cell infected counts k);
//   2. publishes the number of agents it counted, scans the band's counts
//      and gets the band's first output slot from its predecessors by
//      decoupled look-back (bands are handed out in order by an atomic
//      ticket);
//   3. writes start[] for its cells and row_start for its rows;
//   4. reads the records again (now from L2) and, for each agent landing in
//      the band, applies infection (its infection draw against the threshold
//      for the k infected agents of its new cell) or recovery, draws the
//      agent's next-step Philox block (move, and the top byte of the
//      infection draw or the recovery bit its new state needs) and scatters
//      the record to its new slot.
// Per-step S / I / R / new-infection counts are warp-aggregated.
//
// Counters.  32-bit mode: a band whose source rows hold fewer than 65,536
// records keeps one 32-bit word per cell in shared memory: the low half is
// the agent count, then (after the scan) the cell's offset inside the band,
// then the slot cursor; the high half is the infected count.  No half can
// overflow because every value is bounded by the band's record count.  A
// denser band uses two 32-bit counters per cell in a per-CTA slice of global
// memory instead (same steps, exact for any density).  16-bit mode (NarrowCtr
// below): two bytes per cell, so bands are twice as tall for the same shared
// memory; the scan runs one warp per band row and offsets are relative to
// the row; a band whose counts do not fit is redone in the global 32-bit
// counters.
//
// Infection test.  A susceptible agent's record holds the top byte of its
// infection draw u1 for the step; with k infected agents in its new cell it
// is infected iff u1 < T_inf[min(k, K)].  When the threshold lies outside
// the byte's 2^24 values the byte decides; otherwise (about one test in 256)
// the agent's Philox block is recomputed and u1 compared exactly.
#pragma once

#include "amb_internal.cuh"

namespace amb {

constexpr int kBandNT = 1024;
constexpr int kBandCtasPerSm = 1;
constexpr uint32_t kBandSmem = 224u * 1024u;  // dynamic shared memory per CTA (227 KiB minus static)
constexpr uint32_t kMaxBandRows = 32;          // tallest band (source-row tables are static)
constexpr int kMaxSrcRows = kMaxBandRows + 2;
constexpr uint32_t kPackedLimit = 65536;       // records per band for 16-bit halves
constexpr int kU1 = 4;                         // loads per thread and group, pass 1 (two groups in flight)
constexpr int kU2 = 3;                         // loads per thread and group, pass 2 (two groups in flight)

struct BandArgs {
    const uint2 *rec_in;  // {id, word}
    const int32_t *row_in;
    uint2 *rec_out;
    int32_t *row_out;
    int32_t *start;
    uint32_t *wide;  // 2 * H * L words per CTA, or null when n < kPackedLimit and 32-bit shared counters are used
    uint32_t n, L, H, n_bands;
    uint32_t k0, k1, t;  // t = the step executed by this launch
    uint32_t rk0[10], rk1[10];  // Philox round keys of (k0, k1)
    const uint32_t *t_inf;
    uint32_t K, t_rec;
    int64_t *row;       // the step's count row
    int64_t *row_next;  // single-population launches: the next step's count row, cleared here (or null)
    unsigned long long *tickets;
    uint32_t parity;
    uint64_t *status;
    uint32_t epoch;
    uint32_t *err;
    const uint32_t *code_tab;  // precomputed CodeTables (batched steps), or null
};

// Philox4x32-10 block for counter (c0, c1, 0, 0) with the ten round keys
// given (they depend on the key only).
__device__ __forceinline__ U4 philox_rk(uint32_t c0, uint32_t c1, const uint32_t *rk0, const uint32_t *rk1)
{
    constexpr uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
    uint32_t a = c0, b = c1, c = 0u, d = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // high and low halves as two 32-bit multiplies (measured faster here
        // than one widening multiply)
        const uint32_t na = __umulhi(MB, c) ^ b ^ rk0[r];
        const uint32_t nb = MB * c;
        const uint32_t nc = __umulhi(MA, a) ^ d ^ rk1[r];
        const uint32_t nd = MA * a;
        a = na; b = nb; c = nc; d = nd;
    }
    return U4{a, b, c, d};
}

inline void round_keys(uint32_t k0, uint32_t k1, uint32_t *rk0, uint32_t *rk1)
{
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0;
        rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Shared table of the infection thresholds: tinf[k] = T_inf[min(k, K)] for
// k = 0 .. 255 (larger k read the global table).
struct CodeTables {
    uint32_t tinf[256];
};

__device__ __forceinline__ void load_code_tables(CodeTables &ct, const uint32_t *t_inf, uint32_t K)
{
    for (uint32_t i = threadIdx.x; i < 256u; i += blockDim.x) ct.tinf[i] = t_inf[i < K ? i : K];
    __syncthreads();
}

// v + (dp - 1) wrapped on a ring of L sites (v in [0, L), dp in {0, 1, 2})
__device__ __forceinline__ uint32_t wrap_step(uint32_t v, uint32_t dp, uint32_t L)
{
    uint32_t s = v + dp;  // in [0, L + 1], one too large
    s = (s == 0u) ? L : s;
    s = (s == L + 1u) ? 1u : s;
    return s - 1u;
}

// The Moore table as byte tables for one byte permute: byte d of the 8-byte
// value {lo, hi} is dx + 1 (dy + 1) of direction d; byte 0 is 0 in both, so a
// selector whose upper nibbles are 0 leaves the upper result bytes 0.
constexpr uint32_t kDpxLo = 0x00020100u, kDpxHi = 0x02010002u;
constexpr uint32_t kDpyLo = 0x01000000u, kDpyHi = 0x02020201u;
constexpr bool byte_table_matches(uint32_t lo, uint32_t hi, const int *t)
{
    for (int d = 0; d < 8; ++d)
        if ((((d < 4 ? lo : hi) >> (8 * (d & 3))) & 0xFFu) != (uint32_t)(t[d] + 1)) return false;
    return true;
}
static_assert(byte_table_matches(kDpxLo, kDpxHi, kDX) && byte_table_matches(kDpyLo, kDpyHi, kDY),
              "byte tables follow the Moore direction table");

// Record word of an agent at column x whose state (after this step) is st,
// with its draws for step t: the column after its move, the move's dy, and
// the top byte of the infection draw u1 (susceptible) or the recovery bit
// (infected).
__device__ __forceinline__ uint32_t pack_record(const U4 &u, uint32_t st, uint32_t x, uint32_t L, uint32_t t_rec)
{
    const uint32_t d = u.w0 >> 29;
    const uint32_t dpx = __byte_perm(kDpxLo, kDpxHi, d);
    const uint32_t dpy = __byte_perm(kDpyLo, kDpyHi, d);
    const uint32_t w = wrap_step(x, dpx, L) | (st << kAuxStateShift) | (dpy << kAuxDyShift);
    const uint32_t top = (u.w1 >> 24) << kAuxCodeShift;
    const uint32_t rec = (u.w2 < t_rec ? 1u : 0u) << kAuxRecShift;
    return w | (st == AMB_S ? top : (st == AMB_I ? rec : 0u));
}

__device__ __forceinline__ uint32_t record_word(uint32_t id, uint32_t t, uint32_t st, uint32_t x, uint32_t L,
                                                const uint32_t *rk0, const uint32_t *rk1, uint32_t t_rec)
{
    return pack_record(philox_rk(id, t, rk0, rk1), st, x, L, t_rec);
}

// Loads of data that the launch itself never writes (__ldg, the read-only
// path), or, in a persistent launch whose other CTAs wrote it earlier in the
// same launch, through L2 (ld.global.cg: never a stale L1 line).
template <bool kCoherent, class T>
__device__ __forceinline__ T ld_nc(const T *p)
{
    if constexpr (kCoherent)
        return __ldcg(p);
    else
        return __ldg(p);
}

// L2 eviction hints (single-population steps): the cell index start[] and
// the input records after their last read leave L2 first.
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint2 ld_nc_hint(const uint2 *q, uint64_t pol)
{
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(int4 *q, int4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.s32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(q), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w), "l"(pol)
                 : "memory");
}

// ------------------------------------------------------------- counters ---
struct PackedCtr {
    uint32_t *w;  // shared memory
    __device__ __forceinline__ void zero(uint32_t cells) const
    {
        for (uint32_t i = threadIdx.x * 4u; i < cells; i += kBandNT * 4u) {
            if (i + 3u < cells)
                *reinterpret_cast<uint4 *>(&w[i]) = make_uint4(0u, 0u, 0u, 0u);
            else
                for (uint32_t e = i; e < cells; ++e) w[e] = 0u;
        }
    }
    static constexpr bool kNarrow = false;
    // count an agent (and whether it is infected) in cell c; true when the
    // counter overflowed (never, for these counters)
    __device__ __forceinline__ bool add(uint32_t c, bool infected) const
    {
        atomicAdd(&w[c], infected ? 0x10001u : 1u);
        return false;
    }
    __device__ __forceinline__ uint32_t get(uint32_t i) const { return w[i] & 0xFFFFu; }
    __device__ __forceinline__ uint32_t infected(uint32_t c) const { return w[c] >> 16; }
    __device__ __forceinline__ uint32_t take(uint32_t c) const { return atomicAdd(&w[c], 1u) & 0xFFFFu; }
    // four consecutive words i0 .. i0+3 (i0 a multiple of 4); words at or
    // beyond `cells` read as 0 and are not written
    __device__ __forceinline__ void load4(uint32_t i0, uint32_t cells, uint32_t q[4]) const
    {
        if (i0 + 3u < cells) {
            const uint4 v = *reinterpret_cast<const uint4 *>(&w[i0]);
            q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) q[e] = (i0 + e < cells) ? w[i0 + e] : 0u;
        }
    }
    __device__ __forceinline__ static uint32_t count_of(uint32_t q) { return q & 0xFFFFu; }
    // the cells' offsets inside the band replace the counts; the high halves stay
    __device__ __forceinline__ void store4(uint32_t i0, uint32_t cells, const uint32_t q[4], const uint32_t o[4]) const
    {
        if (i0 + 3u < cells) {
            *reinterpret_cast<uint4 *>(&w[i0]) = make_uint4((q[0] & 0xFFFF0000u) | o[0], (q[1] & 0xFFFF0000u) | o[1],
                                                            (q[2] & 0xFFFF0000u) | o[2], (q[3] & 0xFFFF0000u) | o[3]);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (i0 + e < cells) w[i0 + e] = (q[e] & 0xFFFF0000u) | o[e];
        }
    }
};

struct WideCtr {
    uint32_t *cnt, *inf;  // global memory, this CTA's slice
    __device__ __forceinline__ void zero(uint32_t cells) const
    {
        for (uint32_t i = threadIdx.x; i < cells; i += kBandNT) {
            cnt[i] = 0u;
            inf[i] = 0u;
        }
        __threadfence_block();
    }
    static constexpr bool kNarrow = false;
    __device__ __forceinline__ bool add(uint32_t c, bool infected) const
    {
        atomicAdd(&cnt[c], 1u);
        if (infected) atomicAdd(&inf[c], 1u);
        return false;
    }
    __device__ __forceinline__ uint32_t get(uint32_t i) const { return cnt[i]; }
    __device__ __forceinline__ uint32_t infected(uint32_t c) const { return __ldcg(&inf[c]); }
    __device__ __forceinline__ uint32_t take(uint32_t c) const { return atomicAdd(&cnt[c], 1u); }
    __device__ __forceinline__ void load4(uint32_t i0, uint32_t cells, uint32_t q[4]) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e) q[e] = (i0 + e < cells) ? cnt[i0 + e] : 0u;
    }
    __device__ __forceinline__ static uint32_t count_of(uint32_t q) { return q; }
    __device__ __forceinline__ void store4(uint32_t i0, uint32_t cells, const uint32_t *, const uint32_t o[4]) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (i0 + e < cells) cnt[i0 + e] = o[e];
    }
};

// 16-bit counters, two cells per shared word (cell c in the half c & 1 of
// word c >> 1).  While counting, bits [7:0] hold the cell's agents and
// [15:8] its start-of-step infected agents; the scan turns them into the
// cell's offset inside its band row (bits [11:0], then the slot cursor) and
// the infected count (bits [15:12]).  A band fits when no cell holds 256
// agents or 16 infected agents and no band row 4,096 agents; otherwise it is
// redone with 32-bit counters.  Rows are a multiple of 8 cells long.
struct NarrowCtr {
    static constexpr bool kNarrow = true;
    uint32_t *w;  // shared memory
    __device__ __forceinline__ void zero(uint32_t cells) const
    {
        const uint32_t words = (cells + 1u) >> 1;
        for (uint32_t i = threadIdx.x * 4u; i < words; i += kBandNT * 4u) {
            if (i + 3u < words)
                *reinterpret_cast<uint4 *>(&w[i]) = make_uint4(0u, 0u, 0u, 0u);
            else
                for (uint32_t e = i; e < words; ++e) w[e] = 0u;
        }
    }
    // no read-back: a count that wraps (256 agents) lowers the band's sum of
    // agent counts below the number of agents counted, which the scan checks
    // (a carry out of an infected count needs such a wrap first, and adds at
    // most one agent where the wrap took 256)
    __device__ __forceinline__ bool add(uint32_t c, bool infected) const
    {
        atomicAdd(&w[c >> 1], (infected ? 0x101u : 1u) << ((c & 1u) << 4));
        return false;
    }
    // the cell's half before taking a slot: cursor | infected count << 12
    __device__ __forceinline__ uint32_t claim(uint32_t c) const
    {
        const uint32_t sh = (c & 1u) << 4;
        return (atomicAdd(&w[c >> 1], 1u << sh) >> sh) & 0xFFFFu;
    }
};

// The infected count of an agent's new cell, already known.
struct KnownK {
    uint32_t k;
    __device__ __forceinline__ uint32_t infected(uint32_t) const { return k; }
};

struct BandShared {
    CodeTables ct;
    // per source row j of the band: {end of its records in the band's source
    // sequence, slot - sequence index, band row reached with dy = -1, 0, +1
    // (a byte each, 0xFF = outside), grid row}
    uint4 rows[kMaxSrcRows];
    uint32_t warp[kBandNT / 32 + 1];
    uint32_t band, prefix, total;
    uint32_t overflow;                // 16-bit counters: the band does not fit them
    uint32_t rowbase[kMaxBandRows];   // 16-bit counters: each band row's first slot inside the band
    unsigned long long cnt[4];
};

struct Tally {
    uint32_t s, i, r, fresh;
};

// State after this step of an agent whose record (or stage) word is w and
// whose new cell is c of the counters (infected count in the high half).
// The agent's Philox block for step t: round keys from the kernel parameters
// (single-population launches), or derived from the key on the fly (batched
// launches, whose step descriptor sits in shared memory).
template <bool kParamKeys>
__device__ __forceinline__ U4 agent_draws(const BandArgs &a, uint32_t id, uint32_t t)
{
    if constexpr (kParamKeys)
        return philox_rk(id, t, a.rk0, a.rk1);
    else
        return philox(id, t, a.k0, a.k1);
}

// The exact infection test of an agent whose recorded top byte of u1 cannot
// decide: its draw u1 for step t against T_inf[min(k, K)].  Kept out of
// line: it is rare, and inlined its Philox block would raise the register
// demand of the whole record loop.
template <bool kParamKeys>
__device__ __noinline__ bool exact_infection(const BandArgs &a, uint32_t id, uint32_t k)
{
    const U4 q = agent_draws<kParamKeys>(a, id, a.t);
    return q.w1 < a.t_inf[k < a.K ? k : a.K];
}

template <bool kParamKeys, class Ctr>
__device__ __forceinline__ uint32_t new_state(const BandArgs &a, const CodeTables &ct, const Ctr &ctr, uint32_t c,
                                              uint32_t w, uint32_t id, Tally &tl)
{
    uint32_t st = (w >> kAuxStateShift) & 3u;
    if (st == AMB_S) {
        const uint32_t k = ctr.infected(c);
        if (k != 0u) {
            // infected iff u1 < T = T_inf[min(k, K)]; the record holds the top
            // byte of u1: every u1 with that byte is below T, none is, or T
            // lies inside the byte's range and the draw is redone exactly
            const uint32_t T = k < 256u ? ct.tinf[k] : a.t_inf[k < a.K ? k : a.K];
            const uint32_t lo = ((w >> kAuxCodeShift) & 0xFFu) << 24;
            bool hit = (lo | 0xFFFFFFu) < T;
            if (!hit && lo < T) hit = exact_infection<kParamKeys>(a, id, k);
            if (hit) {
                st = AMB_I;
                ++tl.fresh;
            }
        }
    } else if (st == AMB_I) {
        if ((w >> kAuxRecShift) & 1u) st = AMB_R;
    }
    tl.s += 1u;
    tl.i += (st == AMB_I);
    tl.r += (st == AMB_R);
    return st;
}

// Band row a record lands in: byte (dy + 1) of its source row's table (0xFF
// when outside the band, also for the sentinel word 0xFFFFFFFF, whose dy
// field reads 3).
__device__ __forceinline__ uint32_t dest_row(uint32_t tab, uint32_t w)
{
    return __byte_perm(tab, 0u, ((w >> kAuxDyShift) & 3u) | 0x4440u);
}

// Returns false, before writing any record, when the band does not fit
// 16-bit counters (the caller redoes it with 32-bit ones); true otherwise.
template <bool kParamKeys, bool kCoherent, bool kTicketAhead, class Ctr>
__device__ __forceinline__ bool band_body(const BandArgs &a, BandShared &sh, const Ctr &ctr, uint32_t b, uint32_t r0,
                                          uint32_t r1, uint32_t M, Tally &tl)
{
    constexpr bool kNarrow = Ctr::kNarrow;
    const uint32_t L = a.L;
    const uint32_t rows = r1 - r0;
    const uint32_t cells = rows * L;
    const uint32_t tid = threadIdx.x;
    ctr.zero(cells);
    if (tid == 0) {
        sh.total = 0u;
        sh.overflow = 0u;
    }
    __syncthreads();

    // pass 1: agents and start-of-step infected per new cell of the band.
    // A thread takes records v0 + u * kBandNT (u < kU1) per group; two
    // register sets let the loads of the next group fly while the current
    // one is counted.
    {
        uint32_t landed = 0;  // the thread's records that land in the band
        bool ovf = false;     // a 16-bit counter overflowed
        uint32_t j = 0;       // source row of the thread's current record (never decreases)
        uint4 ri = sh.rows[0];
        auto fetch = [&](uint32_t v0, uint32_t(&aux)[kU1], uint32_t(&yy)[kU1]) {
#pragma unroll
            for (int u = 0; u < kU1; ++u) {
                const uint32_t v = v0 + (uint32_t)u * kBandNT;
                aux[u] = 0xFFFFFFFFu;
                yy[u] = 0u;
                if (v < M) {
                    while (ri.x <= v) ri = sh.rows[++j];
                    yy[u] = ri.z;
                    aux[u] = ld_nc<kCoherent>(&a.rec_in[v + ri.y].y);
                }
            }
        };
        auto count = [&](const uint32_t(&aux)[kU1], const uint32_t(&yy)[kU1]) {
#pragma unroll
            for (int u = 0; u < kU1; ++u) {
                const uint32_t w = aux[u];
                if (w == 0xFFFFFFFFu) continue;
                const uint32_t xn = w & kAuxXMask;  // column after the move
                if (xn >= L) {
                    atomicOr(a.err, ERR_RANGE);
                    continue;
                }
                const uint32_t yo = dest_row(yy[u], w);
                if (yo >= rows) continue;  // lands outside the band
                ++landed;
                ovf |= ctr.add(yo * L + xn, ((w >> kAuxStateShift) & 3u) == AMB_I);
            }
        };
        constexpr uint32_t G = kBandNT * kU1;
        uint32_t auxA[kU1], yyA[kU1], auxB[kU1], yyB[kU1];
        fetch(tid, auxA, yyA);
        for (uint32_t v0 = tid; v0 < M; v0 += 2u * G) {
            fetch(v0 + G, auxB, yyB);
            count(auxA, yyA);
            if (v0 + G >= M) break;
            fetch(v0 + 2u * G, auxA, yyA);
            count(auxB, yyB);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) landed += __shfl_xor_sync(0xffffffffu, landed, o);
        if ((tid & 31u) == 0 && landed) atomicAdd(&sh.total, landed);
        if (kNarrow && ovf) sh.overflow = 1u;
    }
    __syncthreads();
    // the band's total is known now: publish it at once, so that successors
    // waiting in look-back see it while this band still scans
    if (tid == 0) lookback_publish(a.status, b, a.epoch, sh.total);
    if (kNarrow && sh.overflow) return false;

    if constexpr (kNarrow) {
        // scan of the band's 16-bit counts, one warp per band row (rows <=
        // 32): (a) row totals (two 16-bit lanes of a word accumulate without
        // carries: a lane adds at most L/64 cells of at most 255 agents,
        // L <= 8192); (b) warp 0 scans them into each row's first slot inside
        // the band and gets the band's first slot P by look-back; (c) each
        // warp turns its row's counts into offsets inside the row and writes
        // the row's start[] = P + row base + offset
        const uint32_t lane = tid & 31u, wid = tid >> 5;
        const uint32_t wpr = L >> 1;  // words per row
        if (wid < rows) {
            const uint32_t *rw = ctr.w + wid * wpr;
            uint32_t acc = 0;
            for (uint32_t i = lane * 4u; i < wpr; i += 128u) {
                const uint4 q = *reinterpret_cast<const uint4 *>(rw + i);
                acc += (q.x & 0x00FF00FFu) + (q.y & 0x00FF00FFu) + (q.z & 0x00FF00FFu) + (q.w & 0x00FF00FFu);
            }
            uint32_t tot = (acc & 0xFFFFu) + (acc >> 16);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            if (lane == 0) {
                sh.rowbase[wid] = tot;
                if (tot >= 4096u) sh.overflow = 1u;  // offsets inside the row need 12 bits
            }
        }
        __syncthreads();
        if (wid == 0) {
            const uint32_t v = lane < rows ? sh.rowbase[lane] : 0u;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += t;
            }
            // T below the agents counted in pass 1: a count wrapped
            const uint32_t T = __shfl_sync(0xffffffffu, incl, 31), counted = sh.total;
            const uint32_t Pb = lookback_wait(a.status, b, a.epoch, counted, a.err);
            if (lane < rows) sh.rowbase[lane] = incl - v;
            if (lane == 0) {
                sh.prefix = Pb;
                if (T != counted) sh.overflow = 1u;
            }
        }
        __syncthreads();
        if (sh.overflow) return false;
        const uint32_t P = sh.prefix;
        if (wid < rows) {
            uint32_t *rw = ctr.w + wid * wpr;
            const uint32_t base = P + sh.rowbase[wid];
            int32_t *srow = a.start + (size_t)(r0 + wid) * L;
            uint32_t run = 0, big = 0;
            // 4 cells (2 words) per lane and step: 16-byte start[] stores,
            // contiguous across the warp
            for (uint32_t i0 = 0; i0 < wpr; i0 += 64u) {
                const uint32_t i = i0 + lane * 2u;
                const bool valid = i < wpr;
                const uint2 q = valid ? *reinterpret_cast<const uint2 *>(rw + i) : make_uint2(0u, 0u);
                const uint32_t n0 = q.x & 0xFFu, n1 = (q.x >> 16) & 0xFFu, n2 = q.y & 0xFFu, n3 = (q.y >> 16) & 0xFFu;
                const uint32_t s4 = (n0 + n1) + (n2 + n3);
                uint32_t incl = s4;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (uint32_t)o) incl += t;
                }
                big |= (q.x | q.y) & 0xF000F000u;  // an infected count >= 16
                const uint32_t o0 = run + incl - s4, o1 = o0 + n0, o2 = o1 + n1, o3 = o2 + n2;
                if (valid) {
                    *reinterpret_cast<uint2 *>(rw + i) = make_uint2(o0 | (o1 << 16) | ((q.x & 0x0F000F00u) << 4),
                                                                    o2 | (o3 << 16) | ((q.y & 0x0F000F00u) << 4));
                    const int4 sv =
                        make_int4((int32_t)(base + o0), (int32_t)(base + o1), (int32_t)(base + o2), (int32_t)(base + o3));
                    if constexpr (kTicketAhead)
                        st_hint(reinterpret_cast<int4 *>(srow + 2u * i), sv, l2_evict_first());
                    else
                        *reinterpret_cast<int4 *>(srow + 2u * i) = sv;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (__any_sync(0xffffffffu, big != 0u) && lane == 0) sh.overflow = 1u;
        }
        if (tid < rows) a.row_out[r0 + tid] = (int32_t)(P + sh.rowbase[tid]);
        if (b == a.n_bands - 1u && tid == 0) {
            a.start[(size_t)L * L] = (int32_t)(P + sh.total);
            a.row_out[L] = (int32_t)(P + sh.total);
        }
        __syncthreads();
        if (sh.overflow) return false;
    } else {
        // scan of the band's counts: every warp owns a run of consecutive cells
        // (groups of four); (a) warp totals, (b) warp 0 scans them and gets the
        // band's first slot P by look-back, (c) every warp turns its counts into
        // offsets and writes the cell index start[] = P + offset
        constexpr uint32_t kWarps = kBandNT / 32;
        static_assert(kWarps <= 32, "one warp scans the warp totals");
        const uint32_t lane = tid & 31u, wid = tid >> 5;
        const uint32_t quads = (cells + 3u) >> 2, qpw = (quads + kWarps - 1u) / kWarps;
        const uint32_t q0 = wid * qpw, q1 = min(q0 + qpw, quads);
        {
            uint32_t part = 0;
            for (uint32_t q = q0 + lane; q < q1; q += 32u) {
                uint32_t c[4];
                ctr.load4(q * 4u, cells, c);
                part += Ctr::count_of(c[0]) + Ctr::count_of(c[1]) + Ctr::count_of(c[2]) + Ctr::count_of(c[3]);
            }
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == 0) sh.warp[wid] = part;
        }
        __syncthreads();
        if (wid == 0) {
            const uint32_t v = lane < kWarps ? sh.warp[lane] : 0u;
            uint32_t incl = v;
    #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += t;
            }
            const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t P = lookback_wait(a.status, b, a.epoch, T, a.err);
            if (lane < kWarps) sh.warp[lane] = incl - v;
            if (lane == 0) {
                sh.prefix = P;
                sh.total = T;
            }
        }
        __syncthreads();
        const uint32_t P = sh.prefix;
        {
            int32_t *start_band = a.start + (size_t)r0 * L;
            const bool vec = (((size_t)r0 * L) & 3u) == 0;  // 16-byte aligned start[] stores
            uint32_t run = sh.warp[wid];
            for (uint32_t qb = q0; qb < q1; qb += 32u) {
                const uint32_t q = qb + lane, i0 = q * 4u;
                uint32_t c[4] = {0u, 0u, 0u, 0u};
                if (q < q1) ctr.load4(i0, cells, c);
                const uint32_t n0 = Ctr::count_of(c[0]), n1 = Ctr::count_of(c[1]), n2 = Ctr::count_of(c[2]);
                const uint32_t s4 = n0 + n1 + n2 + Ctr::count_of(c[3]);
                uint32_t incl = s4;
    #pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (uint32_t)o) incl += t;
                }
                uint32_t off[4];
                off[0] = run + incl - s4;
                off[1] = off[0] + n0;
                off[2] = off[1] + n1;
                off[3] = off[2] + n2;
                if (q < q1) {
                    ctr.store4(i0, cells, c, off);
                    if (vec && i0 + 3u < cells) {
                        *reinterpret_cast<int4 *>(start_band + i0) =
                            make_int4((int32_t)(P + off[0]), (int32_t)(P + off[1]), (int32_t)(P + off[2]),
                                      (int32_t)(P + off[3]));
                    } else {
    #pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (i0 + e < cells) start_band[i0 + e] = (int32_t)(P + off[e]);
                    }
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        __syncthreads();
        // row starts (before pass 2 moves the offsets on)
        for (uint32_t r = tid; r < rows; r += kBandNT) a.row_out[r0 + r] = (int32_t)(P + ctr.get(r * L));
        if (b == a.n_bands - 1u && tid == 0) {
            a.start[(size_t)L * L] = (int32_t)(P + sh.total);
            a.row_out[L] = (int32_t)(P + sh.total);
        }
        __syncthreads();
    }
    const uint32_t P = sh.prefix;

    // the band this CTA takes next (sir_band_kernel reads it after the
    // band): its ticket's latency hides behind pass 2
    if constexpr (kTicketAhead)
        if (tid == 0) sh.band = (uint32_t)atomicAdd(&a.tickets[a.parity], 1ull);

    // pass 2: transitions, next draws, scatter (the records come from L2),
    // with the loads of the next group in flight as in pass 1
    {
        uint32_t j = 0;
        uint4 ri = sh.rows[0];
        auto fetch = [&](uint32_t v0, uint32_t(&ids)[kU2], uint32_t(&aux)[kU2], uint32_t(&yy)[kU2]) {
#pragma unroll
            for (int u = 0; u < kU2; ++u) {
                const uint32_t v = v0 + (uint32_t)u * kBandNT;
                aux[u] = 0xFFFFFFFFu;
                ids[u] = 0u;
                yy[u] = 0xFFFFFFFFu;
                if (v < M) {
                    while (ri.x <= v) ri = sh.rows[++j];
                    yy[u] = ri.z;
                    uint2 rv;
                    if constexpr (kTicketAhead && !kCoherent)
                        rv = ld_nc_hint(&a.rec_in[v + ri.y], l2_evict_first());  // the record's last read
                    else
                        rv = ld_nc<kCoherent>(&a.rec_in[v + ri.y]);
                    ids[u] = rv.x;
                    aux[u] = rv.y;
                }
            }
        };
        auto update = [&](const uint32_t(&ids)[kU2], const uint32_t(&aux)[kU2], const uint32_t(&yy)[kU2]) {
            // in phases over the group's records, so that their Philox
            // blocks are independent instruction streams
            uint32_t slot[kU2], st[kU2];
            bool ok[kU2];
#pragma unroll
            for (int u = 0; u < kU2; ++u) {
                const uint32_t w = aux[u];
                const uint32_t xn = w & kAuxXMask;
                const uint32_t yo = dest_row(yy[u], w);
                ok[u] = (xn < L) && (yo < rows);  // the sentinel word lands nowhere
                const uint32_t c = yo * L + xn;
                st[u] = 0u;
                slot[u] = 0u;
                if (ok[u]) {
                    if constexpr (kNarrow) {
                        // one atomic gives the slot cursor and the infected count
                        const uint32_t half = ctr.claim(c);
                        st[u] = new_state<kParamKeys>(a, sh.ct, KnownK{half >> 12}, c, w, ids[u], tl);
                        slot[u] = P + sh.rowbase[yo] + (half & 0xFFFu);
                    } else {
                        st[u] = new_state<kParamKeys>(a, sh.ct, ctr, c, w, ids[u], tl);
                        slot[u] = P + ctr.take(c);
                    }
                }
                if (ok[u] && slot[u] >= a.n) {
                    atomicOr(a.err, ERR_OVERFLOW);
                    ok[u] = false;
                }
            }
            U4 r[kU2];
#pragma unroll
            for (int u = 0; u < kU2; ++u) r[u] = agent_draws<kParamKeys>(a, ids[u], a.t + 1u);
#pragma unroll
            for (int u = 0; u < kU2; ++u) {
                if (!ok[u]) continue;
                const uint2 rec = make_uint2(ids[u], pack_record(r[u], st[u], aux[u] & kAuxXMask, L, a.t_rec));
                a.rec_out[slot[u]] = rec;
            }
        };
        constexpr uint32_t G = kBandNT * kU2;
        uint32_t idsA[kU2], auxA[kU2], yyA[kU2], idsB[kU2], auxB[kU2], yyB[kU2];
        fetch(tid, idsA, auxA, yyA);
        for (uint32_t v0 = tid; v0 < M; v0 += 2u * G) {
            fetch(v0 + G, idsB, auxB, yyB);
            update(idsA, auxA, yyA);
            if (v0 + G >= M) break;
            fetch(v0 + 2u * G, idsA, auxA, yyA);
            update(idsB, auxB, yyB);
        }
    }
    __syncthreads();
    return true;
}

// All threads: band b of the step described by `a` (its source-row tables,
// then band_body with shared-memory or, for very dense bands, global
// counters).  kTicketAhead: thread 0 draws the ticket of the CTA's next band
// into sh.band when pass 2 starts.  kNarrow: 16-bit shared counters (rows a
// multiple of 8 cells, at most 8192), else 32-bit ones.
template <bool kParamKeys, bool kCoherent, bool kTicketAhead = false, bool kNarrow = false>
__device__ __forceinline__ void process_band(const BandArgs &a, BandShared &sh, uint32_t *band_smem,
                                             uint32_t *wide_slice, uint32_t b, Tally &tl)
{
    const uint32_t L = a.L, tid = threadIdx.x;
    const bool single = (a.n_bands == 1);
    // bands of floor / ceil(L / n_bands) rows
    const uint32_t r0 = (uint32_t)(((uint64_t)b * L) / a.n_bands);
    const uint32_t r1 = (uint32_t)(((uint64_t)(b + 1u) * L) / a.n_bands);
    // source rows r0-1 .. r1 (all rows, once, when one band covers the grid)
    const uint32_t nsrc = single ? L : (r1 - r0) + 2u;
    uint32_t len = 0, beg = 0, y = 0;
    if (tid < nsrc) {
        y = single ? tid : (r0 + L - 1u + tid) % L;
        const int32_t b0 = ld_nc<kCoherent>(&a.row_in[y]), b1 = ld_nc<kCoherent>(&a.row_in[y + 1]);
        if (b0 >= 0 && b1 >= b0 && (uint32_t)b1 <= a.n) {
            beg = (uint32_t)b0;
            len = (uint32_t)(b1 - b0);
        } else {
            atomicOr(a.err, ERR_RANGE);  // a corrupt row table: the row is skipped
        }
    }
    uint32_t M;
    const uint32_t off = block_exclusive_scan<kBandNT>(len, sh.warp, &M);
    if (tid < nsrc) {
        // record v of the band's source sequence with off <= v < off + len
        // sits at slot v + (beg - off) (modulo 2^32)
        uint32_t tab = 0xFF000000u;  // byte 3: the dy field 3 of the sentinel word lands nowhere
        for (uint32_t dp = 0; dp < 3u; ++dp) {
            const uint32_t yo = wrap_step(y, dp, L) - r0;  // wraps above 0xFF when outside
            tab |= (yo < r1 - r0 ? yo : 0xFFu) << (8u * dp);
        }
        sh.rows[tid] = make_uint4(off + len, beg - off, tab, y);
    }
    __syncthreads();
    if constexpr (kNarrow) {
        // 16-bit counters; a band that does not fit them is redone with
        // 32-bit counters in global memory (allocated with the narrow band
        // shape: the shared array holds only 2 bytes per cell)
        if (wide_slice == nullptr) {
            if (tid == 0) atomicOr(a.err, ERR_OVERFLOW);
            return;
        }
        if (!band_body<kParamKeys, kCoherent, kTicketAhead>(a, sh, NarrowCtr{band_smem}, b, r0, r1, M, tl))
            band_body<kParamKeys, kCoherent, kTicketAhead>(a, sh, WideCtr{wide_slice, wide_slice + (size_t)a.H * L}, b,
                                                           r0, r1, M, tl);
    } else {
        if (M < kPackedLimit || wide_slice == nullptr)
            band_body<kParamKeys, kCoherent, kTicketAhead>(a, sh, PackedCtr{band_smem}, b, r0, r1, M, tl);
        else
            band_body<kParamKeys, kCoherent, kTicketAhead>(a, sh, WideCtr{wide_slice, wide_slice + (size_t)a.H * L}, b,
                                                           r0, r1, M, tl);
    }
}

// All threads: add the block's tally to row[0..3] and clear it.
__device__ __forceinline__ void flush_tally(BandShared &sh, Tally &tl, int64_t *row)
{
    const uint32_t tid = threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tl.s += __shfl_down_sync(0xffffffffu, tl.s, o);
        tl.i += __shfl_down_sync(0xffffffffu, tl.i, o);
        tl.r += __shfl_down_sync(0xffffffffu, tl.r, o);
        tl.fresh += __shfl_down_sync(0xffffffffu, tl.fresh, o);
    }
    if ((tid & 31u) == 0) {
        tl.s -= tl.i + tl.r;
        if (tl.s) atomicAdd(&sh.cnt[0], (unsigned long long)tl.s);
        if (tl.i) atomicAdd(&sh.cnt[1], (unsigned long long)tl.i);
        if (tl.r) atomicAdd(&sh.cnt[2], (unsigned long long)tl.r);
        if (tl.fresh) atomicAdd(&sh.cnt[3], (unsigned long long)tl.fresh);
    }
    __syncthreads();
    if (tid < 4) {
        if (sh.cnt[tid]) atomicAdd(reinterpret_cast<unsigned long long *>(&row[tid]), sh.cnt[tid]);
        sh.cnt[tid] = 0ull;
    }
    tl = Tally{0u, 0u, 0u, 0u};
    __syncthreads();
}

}  // namespace amb
