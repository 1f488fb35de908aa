// amb_common.cuh -- shared device/host helpers of the CUDA library.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) written from the
// published round function; Moore direction table; bounded decoupled
// look-back for single-pass scans (Merrill & Garland, "Single-pass parallel
// prefix scan with decoupled look-back", 2016); status helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "amb.h"

namespace amb {

// ---------------------------------------------------------------- status ---
amb_status fail(amb_status st, const char *fmt, ...);
void clear_error();

#define AMB_TRY_CUDA(call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::amb::fail(AMB_ECUDA, "%s failed: %s (%s:%d)", #call,              \
                               cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)

#define AMB_TRY(expr)                        \
    do {                                     \
        amb_status s_ = (expr);              \
        if (s_ != AMB_OK) return s_;         \
    } while (0)

// Device error word bits (sticky per population / per call).
enum : uint32_t {
    ERR_TIMEOUT = 1u,    // a bounded spin ran out
    ERR_RANGE = 2u,      // a coordinate / state outside its domain was met
    ERR_OVERFLOW = 4u,   // a capacity bound was exceeded
};

// ---------------------------------------------------------------- philox ---
struct U4 {
    uint32_t w0, w1, w2, w3;
};

// One Philox4x32-10 block for counter (c0, c1, 0, 0) and key (k0, k1).
__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
    constexpr uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
    uint32_t a = c0, b = c1, c = 0u, d = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t pa = (uint64_t)MA * a;
        const uint64_t pb = (uint64_t)MB * c;
        const uint32_t na = (uint32_t)(pb >> 32) ^ b ^ k0;
        const uint32_t nb = (uint32_t)pb;
        const uint32_t nc = (uint32_t)(pa >> 32) ^ d ^ k1;
        const uint32_t nd = (uint32_t)pa;
        a = na; b = nb; c = nc; d = nd;
        k0 += WA;
        k1 += WB;
    }
    return U4{a, b, c, d};
}

constexpr uint32_t kInitStep = 0xFFFFFFFFu;

// hi32(u * n): uniform integer in [0, n) from one 32-bit word.
__host__ __device__ __forceinline__ uint32_t below(uint32_t u, uint32_t n)
{
    return (uint32_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

// ----------------------------------------------------------- moore table ---
// Direction d (top three bits of the move word) -> (dx, dy):
//   0 (-1,-1) 1 (0,-1) 2 (1,-1) 3 (-1,0) 4 (1,0) 5 (-1,1) 6 (0,1) 7 (1,1)
// Packed as 2-bit fields of (delta + 1).
constexpr int kDX[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
constexpr int kDY[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
constexpr uint32_t pack_dirs(const int *t)
{
    uint32_t v = 0;
    for (int d = 0; d < 8; ++d) v |= (uint32_t)(t[d] + 1) << (2 * d);
    return v;
}
constexpr uint32_t kPackDX = pack_dirs(kDX);
constexpr uint32_t kPackDY = pack_dirs(kDY);

__host__ __device__ __forceinline__ int dir_dx(uint32_t d) { return (int)((kPackDX >> (2 * d)) & 3u) - 1; }
__host__ __device__ __forceinline__ int dir_dy(uint32_t d) { return (int)((kPackDY >> (2 * d)) & 3u) - 1; }

// v + delta on a ring of L sites, v in [0, L), delta in {-1, 0, 1}.
__host__ __device__ __forceinline__ int32_t ring_add(int32_t v, int delta, int32_t L)
{
    int32_t s = v + delta;
    s = (s < 0) ? s + L : s;
    s = (s >= L) ? s - L : s;
    return s;
}

// ------------------------------------------------------ decoupled lookback ---
// Tile status word: [63:34] epoch (never 0 for a live launch), [33:32] flag,
// [31:0] value.  flag 1 = tile aggregate, 2 = inclusive prefix.
constexpr uint64_t kFlagAgg = 1ull, kFlagPrefix = 2ull;
constexpr uint64_t kSpinLimitNs = 2000000000ull;  // give up a wait after 2 s

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t error_word(const uint32_t *err)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(err) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t status_word(uint32_t epoch, uint64_t flag, uint32_t v)
{
    return ((uint64_t)epoch << 34) | (flag << 32) | (uint64_t)v;
}

__device__ __forceinline__ void status_store(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t status_load(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Publish the aggregate of tile `tile`, then walk back over the predecessors
// until an inclusive prefix is found; publish this tile's inclusive prefix and
// return the exclusive prefix.  Called by ONE thread.  Tiles are handed out in
// increasing order by an atomic ticket, so every predecessor is already
// running or finished and each wait ends; the spin is still bounded: after
// kSpinLimitNs of waiting, or as soon as another waiter has given up, the
// error word gets ERR_TIMEOUT and the walk stops (the result is then wrong,
// and the host reports AMB_ETIMEOUT).
__device__ __forceinline__ uint32_t lookback_exclusive(uint64_t *status, uint32_t tile, uint32_t epoch,
                                                       uint32_t aggregate, uint32_t *err)
{
    if (tile == 0) {
        status_store(&status[0], status_word(epoch, kFlagPrefix, aggregate));
        return 0u;
    }
    status_store(&status[tile], status_word(epoch, kFlagAgg, aggregate));
    uint32_t excl = 0;
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    unsigned backoff = 8;
    uint64_t t0 = 0;
    while (j >= 0) {
        const uint64_t s = status_load(&status[j]);
        const uint32_t ep = (uint32_t)(s >> 34);
        const uint64_t fl = (s >> 32) & 3ull;
        if (ep == epoch && fl != 0ull) {
            excl += (uint32_t)s;
            if (fl == kFlagPrefix) break;
            --j;
            continue;
        }
        if (spins == 0) t0 = global_ns();
        if ((++spins & 63u) == 0u) {
            if ((error_word(err) & ERR_TIMEOUT) || global_ns() - t0 > kSpinLimitNs) {
                atomicOr(err, ERR_TIMEOUT);
                break;
            }
        }
        __nanosleep(backoff);
        if (backoff < 256) backoff <<= 1;
    }
    status_store(&status[tile], status_word(epoch, kFlagPrefix, excl + aggregate));
    return excl;
}

// One thread: publish the tile's aggregate (tile 0: its inclusive prefix),
// so that successors can walk past it before it knows its own prefix.
__device__ __forceinline__ void lookback_publish(uint64_t *status, uint32_t tile, uint32_t epoch, uint32_t aggregate)
{
    status_store(&status[tile], status_word(epoch, tile == 0 ? kFlagPrefix : kFlagAgg, aggregate));
}

// One warp (all 32 lanes), after lookback_publish of the same tile: walk
// back 32 predecessors at a time (one ballot per 32 status words), publish
// the inclusive prefix and return the exclusive prefix (all lanes).
// Bounded like lookback_exclusive (timer + shared error word).
__device__ __forceinline__ uint32_t lookback_wait(uint64_t *status, uint32_t tile, uint32_t epoch, uint32_t aggregate,
                                                  uint32_t *err)
{
    const uint32_t lane = threadIdx.x & 31u;
    if (tile == 0) return 0u;
    uint32_t excl = 0;
    int64_t base = (int64_t)tile - 1;
    uint32_t spins = 0;
    uint64_t t0 = 0;
    unsigned backoff = 16;
    while (base >= 0) {
        const int64_t j = base - (int64_t)lane;
        const uint64_t s = (j >= 0) ? status_load(&status[j]) : status_word(epoch, kFlagPrefix, 0u);
        const uint64_t fl = (s >> 32) & 3ull;
        const bool ready = ((uint32_t)(s >> 34) == epoch) && fl != 0ull;
        const uint32_t pm = __ballot_sync(0xffffffffu, ready && fl == kFlagPrefix);
        const uint32_t rm = __ballot_sync(0xffffffffu, ready);
        const uint32_t last = pm ? (uint32_t)(__ffs(pm) - 1) : 31u;
        const uint32_t need = (last == 31u) ? 0xffffffffu : ((1u << (last + 1u)) - 1u);
        if ((rm & need) == need) {
            uint32_t v = (lane <= last) ? (uint32_t)s : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            excl += v;
            if (pm) break;
            base -= 32;
            continue;
        }
        if (spins == 0) t0 = global_ns();
        bool give_up = false;
        if ((++spins & 15u) == 0u)
            give_up = (error_word(err) & ERR_TIMEOUT) || (global_ns() - t0 > kSpinLimitNs);
        give_up = __shfl_sync(0xffffffffu, give_up, 0);
        if (give_up) {
            if (lane == 0) atomicOr(err, ERR_TIMEOUT);
            break;
        }
        __nanosleep(backoff);
        if (backoff < 256) backoff <<= 1;
    }
    if (lane == 0) status_store(&status[tile], status_word(epoch, kFlagPrefix, excl + aggregate));
    return excl;
}

// One warp: lookback_publish by lane 0, then lookback_wait.
__device__ __forceinline__ uint32_t warp_lookback(uint64_t *status, uint32_t tile, uint32_t epoch, uint32_t aggregate,
                                                  uint32_t *err)
{
    if ((threadIdx.x & 31u) == 0) lookback_publish(status, tile, epoch, aggregate);
    return lookback_wait(status, tile, epoch, aggregate, err);
}

// ------------------------------------------------------------ block scan ---
// Exclusive scan of one uint32 per thread over a block of NT threads; returns
// the exclusive prefix and writes the block total to *total (all threads).
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *smem_warp /* NT/32 + 1 */,
                                                         uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        constexpr int NW = NT / 32;
        uint32_t w = (lane < NW) ? smem_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) smem_warp[lane] = wi - w;
        if (lane == NW - 1) smem_warp[NW] = wi;
    }
    __syncthreads();
    const uint32_t res = smem_warp[warp] + incl - v;
    *total = smem_warp[NT / 32];
    __syncthreads();
    return res;
}

// ------------------------------------------------------------- host side ---
// Threshold table of the SIR step (see amb_sir_thresholds in amb.h).
amb_status host_thresholds(double beta, double gamma, uint32_t cap, uint32_t *t_inf, uint32_t *K,
                           uint32_t *t_rec);

// Multiprocessor count of the current device (queried once per device).
unsigned device_sms();

// Blocks for `work` items at `per_block` per block, at most `per_sm` blocks
// per multiprocessor of the current device.
inline unsigned grid_for(uint64_t work, unsigned per_block, unsigned per_sm = 64u)
{
    uint64_t g = (work + per_block - 1) / per_block;
    const uint64_t cap = (uint64_t)device_sms() * per_sm;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace amb
