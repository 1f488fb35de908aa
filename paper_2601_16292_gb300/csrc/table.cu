// table.cu -- the view API over a device-resident columnar table (paper
// Sec. 3.1 and 3.3): full-population views (one elementwise kernel over a
// column), filtered views (an order-preserving stream compaction of the ids
// whose value satisfies a predicate: per-thread predicate bits, warp-free
// popc counts, a block scan and a decoupled look-back across tiles) and
// scatter views (id lists in which ids repeat; updates through them use
// atomics, so contributions of repeated ids accumulate).  A view's length
// lives on the device, so chains of view operations run without host
// synchronisation; every kernel reads it there.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "amb_internal.cuh"

using namespace amb;

namespace {

struct Column {
    std::string name;
    amb_dtype dtype;
    void *ptr = nullptr;  // int32[n] or uint8[n rounded up to 4]
};

}  // namespace

struct amb_table {
    uint32_t n = 0;
    cudaStream_t stream = nullptr;
    std::vector<Column> cols;
    uint32_t *err = nullptr;
    int live_views = 0;
    // where() scratch, made on first use: predicate words, per-tile counts
    // and their exclusive scan
    uint32_t *where_bits = nullptr;
    int32_t *where_cnt = nullptr, *where_off = nullptr;
    uint32_t *where_done = nullptr;  // blocks of the flag launch that finished (the last resets it)
    uint32_t where_tiles = 0;        // write tiles the scratch holds
};

struct amb_log {
    amb_table *t = nullptr;
    uint32_t capacity = 0, count = 0;
    int32_t *ids = nullptr, *cols = nullptr;
    int64_t *vals = nullptr;
    // per column: the number of the winning record per row (-1 = none), when
    // used.  Records are numbered across flushes (base + index), so words
    // left by earlier flushes never match and need no reset.
    std::vector<int32_t *> win;
    std::vector<bool> used;      // columns recorded since the last flush
    uint32_t base = 0;           // number of the first record of the next flush
};

struct amb_view {
    amb_table *t = nullptr;
    int32_t *ids = nullptr;   // capacity entries
    uint32_t *count = nullptr;  // device
    uint32_t capacity = 0;
    bool unique = false;      // filtered views list every id at most once
};

namespace {

// ------------------------------------------------------------ operations ---
template <int OP, class T>
__device__ __forceinline__ T apply(T a, T b)
{
    if constexpr (OP == AMB_OP_SET) return b;
    if constexpr (OP == AMB_OP_ADD) return (T)(a + b);
    if constexpr (OP == AMB_OP_SUB) return (T)(a - b);
    if constexpr (OP == AMB_OP_MUL) return (T)(a * b);
    if constexpr (OP == AMB_OP_MIN) return a < b ? a : b;
    return a > b ? a : b;
}

// int32 arithmetic wraps: do it on the unsigned representation
template <int OP>
__device__ __forceinline__ int32_t apply_i32(int32_t a, int32_t b)
{
    if constexpr (OP == AMB_OP_MIN || OP == AMB_OP_MAX || OP == AMB_OP_SET) return apply<OP, int32_t>(a, b);
    return (int32_t)apply<OP, uint32_t>((uint32_t)a, (uint32_t)b);
}

template <int OP>
__device__ __forceinline__ uint8_t apply_u8(uint8_t a, uint8_t b)
{
    return apply<OP, uint8_t>(a, b);
}

template <int CMP>
__device__ __forceinline__ bool compare(int64_t v, int64_t s)
{
    if constexpr (CMP == AMB_CMP_EQ) return v == s;
    if constexpr (CMP == AMB_CMP_NE) return v != s;
    if constexpr (CMP == AMB_CMP_LT) return v < s;
    if constexpr (CMP == AMB_CMP_LE) return v <= s;
    if constexpr (CMP == AMB_CMP_GT) return v > s;
    return v >= s;
}

constexpr int kMapNT = 256;
constexpr int kMaxLogCols = 64;  // columns a buffered-write log can address

// full-population view, scalar operand: 4 int32 (or 16 uint8) per 16-byte access
template <int OP>
__global__ void __launch_bounds__(kMapNT) map_i32_kernel(int32_t *__restrict__ c, uint32_t n, int32_t s)
{
    const uint32_t nv = n / 4u;
    int4 *v = reinterpret_cast<int4 *>(c);
    for (uint32_t i = blockIdx.x * kMapNT + threadIdx.x; i < nv; i += gridDim.x * kMapNT) {
        int4 q = v[i];
        q.x = apply_i32<OP>(q.x, s);
        q.y = apply_i32<OP>(q.y, s);
        q.z = apply_i32<OP>(q.z, s);
        q.w = apply_i32<OP>(q.w, s);
        v[i] = q;
    }
    for (uint32_t i = nv * 4u + blockIdx.x * kMapNT + threadIdx.x; i < n; i += gridDim.x * kMapNT)
        c[i] = apply_i32<OP>(c[i], s);
}

template <int OP>
__global__ void __launch_bounds__(kMapNT) map_u8_kernel(uint8_t *__restrict__ c, uint32_t n, uint8_t s)
{
    const uint32_t nv = n / 16u;
    uint4 *v = reinterpret_cast<uint4 *>(c);
    for (uint32_t i = blockIdx.x * kMapNT + threadIdx.x; i < nv; i += gridDim.x * kMapNT) {
        uint4 q = v[i];
        uint32_t *w = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t r = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                r |= (uint32_t)apply_u8<OP>((uint8_t)(w[k] >> (8 * b)), s) << (8 * b);
            w[k] = r;
        }
        v[i] = q;
    }
    for (uint32_t i = nv * 16u + blockIdx.x * kMapNT + threadIdx.x; i < n; i += gridDim.x * kMapNT)
        c[i] = apply_u8<OP>(c[i], s);
}

// full-population view, column operand (element by element)
template <int OP, class D, class S>
__global__ void __launch_bounds__(kMapNT) map_col_kernel(D *__restrict__ d, const S *__restrict__ src, uint32_t n)
{
    for (uint32_t i = blockIdx.x * kMapNT + threadIdx.x; i < n; i += gridDim.x * kMapNT) {
        if constexpr (sizeof(D) == 4)
            d[i] = apply_i32<OP>(d[i], (int32_t)src[i]);
        else
            d[i] = apply_u8<OP>(d[i], (uint8_t)src[i]);
    }
}

// ---------------------------------------------------------------- where ---
// Order-preserving compaction in two streaming launches with no chain between
// tiles, over the rows of a column or, for a view of a view, over the entries
// of a view's id list (the column read through the ids; list order kept).
// (1) Every block reads a span, 8 consecutive positions per thread and span
// row (2 x 16 bytes of int32 values or ids, 8 bytes of uint8 values), writes
// their predicate bits as one byte to shared memory, so that the block's
// shared bytes are the span's bitmap in position order, stores the bitmap and
// the count of every write tile (kWhereTile positions); the last block to
// finish scans the counts.  (2) One block per write tile turns its bitmap
// into ids, each warp writing the selected positions of each 32-position word
// as one contiguous run.
constexpr int kWhereNT = 512;
constexpr uint32_t kWhereTile = 32u * kWhereNT;        // positions per write tile: one predicate word per thread
constexpr uint32_t kWhereWords = kWhereTile / 32u;
constexpr int kWhereRowsI32 = 8;   // span rows over int32 values or over a list
constexpr int kWhereRowsU8 = 16;   // span rows over uint8 values
template <class T, bool kList>
struct WhereSpan {
    static constexpr uint32_t kRows = (kList || sizeof(T) == 4) ? kWhereRowsI32 : kWhereRowsU8;  // 8 positions per thread each
    static constexpr uint32_t kBytes = kRows * kWhereNT;          // bitmap bytes of a span
    static constexpr uint32_t kItems = kBytes * 8u;               // positions of a span
    static constexpr uint32_t kTiles = kItems / kWhereTile;       // write tiles per span
};

// predicate bits of positions i .. i + 7 (bit k: position i + k); the value at
// position p is c[p], or c[in[p]] over a list
template <int CMP, class T, bool kList>
__device__ __forceinline__ uint32_t where_bits8(const T *__restrict__ c, const int32_t *__restrict__ in, uint32_t i,
                                                uint32_t n, int64_t s)
{
    uint32_t f = 0;
    if (i + 8u <= n) {
        if constexpr (kList) {
            const int4 a = *reinterpret_cast<const int4 *>(in + i), b = *reinterpret_cast<const int4 *>(in + i + 4);
            const int32_t id[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            T v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = c[id[k]];
#pragma unroll
            for (int k = 0; k < 8; ++k) f |= (uint32_t)compare<CMP>((int64_t)v[k], s) << k;
        } else if constexpr (sizeof(T) == 4) {
            const int4 a = *reinterpret_cast<const int4 *>(c + i), b = *reinterpret_cast<const int4 *>(c + i + 4);
            const int32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int k = 0; k < 8; ++k) f |= (uint32_t)compare<CMP>((int64_t)v[k], s) << k;
        } else {
            const uint2 a = *reinterpret_cast<const uint2 *>(c + i);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                f |= (uint32_t)compare<CMP>((int64_t)(((k < 4 ? a.x : a.y) >> (8 * (k & 3))) & 0xFFu), s) << k;
        }
    } else {
        for (uint32_t k = 0; k < 8u; ++k)
            if (i + k < n && compare<CMP>((int64_t)c[kList ? (uint32_t)in[i + k] : i + k], s)) f |= 1u << k;
    }
    return f;
}

// n positions, or *n_dev of them when n_dev is given (a view's length)
template <int CMP, class T, bool kList>
__global__ void __launch_bounds__(kWhereNT) where_flags_kernel(const T *__restrict__ c, const int32_t *__restrict__ in,
                                                               uint32_t n, const uint32_t *__restrict__ n_dev,
                                                               int64_t s, uint32_t *__restrict__ bits,
                                                               int32_t *__restrict__ cnt, int32_t *__restrict__ off,
                                                               uint32_t n_tiles, uint32_t *__restrict__ done,
                                                               uint32_t *__restrict__ count)
{
    using Sp = WhereSpan<T, kList>;
    __shared__ __align__(16) uint8_t s_map[Sp::kBytes];
    __shared__ uint32_t s_sum[Sp::kTiles][kWhereNT / 32];
    __shared__ uint32_t s_warp[kWhereNT / 32 + 1];
    __shared__ bool s_last;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const uint32_t len = n_dev ? *n_dev : n;
    const uint32_t span0 = blockIdx.x * Sp::kItems;
#pragma unroll 4
    for (uint32_t r = 0; r < Sp::kRows; ++r)
        s_map[r * kWhereNT + tid] =
            (uint8_t)where_bits8<CMP, T, kList>(c, in, span0 + (r * kWhereNT + tid) * 8u, len, s);
    __syncthreads();
    // word tid + k kWhereNT of the span is word tid of its write tile k
    const uint32_t *wmap = reinterpret_cast<const uint32_t *>(s_map);
    const uint32_t tile0 = blockIdx.x * Sp::kTiles;
#pragma unroll
    for (uint32_t k = 0; k < Sp::kTiles; ++k) {
        const uint32_t w = wmap[k * kWhereNT + tid];
        if (tile0 + k < n_tiles) bits[(size_t)(tile0 + k) * kWhereWords + tid] = w;
        uint32_t p = __popc(w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if (lane == 0) s_sum[k][wid] = p;
    }
    __syncthreads();
    if (tid < Sp::kTiles && tile0 + tid < n_tiles) {
        uint32_t p = 0;
        for (uint32_t w = 0; w < kWhereNT / 32; ++w) p += s_sum[tid][w];
        cnt[tile0 + tid] = (int32_t)p;
    }
    // the last block to finish scans every tile's count
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(done, 1u) == gridDim.x - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // thread i scans a segment of `per` counts (all of them loaded at once
    // when per <= kFast)
    constexpr uint32_t kFast = 16;
    const uint32_t per = (n_tiles + kWhereNT - 1u) / kWhereNT, j0 = min(tid * per, n_tiles), j1 = min(j0 + per, n_tiles);
    uint32_t total;
    if (per <= kFast) {
        uint32_t val[kFast], part = 0;
#pragma unroll
        for (uint32_t q = 0; q < kFast; ++q) {
            val[q] = (j0 + q < j1) ? (uint32_t)__ldcg(cnt + j0 + q) : 0u;
            part += val[q];
        }
        uint32_t run = block_exclusive_scan<kWhereNT>(part, s_warp, &total);
#pragma unroll
        for (uint32_t q = 0; q < kFast; ++q) {
            if (j0 + q < j1) off[j0 + q] = (int32_t)run;
            run += val[q];
        }
    } else {
        uint32_t part = 0;
        for (uint32_t j = j0; j < j1; ++j) part += (uint32_t)__ldcg(cnt + j);
        uint32_t run = block_exclusive_scan<kWhereNT>(part, s_warp, &total);
        for (uint32_t j = j0; j < j1; ++j) {
            off[j] = (int32_t)run;
            run += (uint32_t)__ldcg(cnt + j);
        }
    }
    if (tid == 0) {
        off[n_tiles] = (int32_t)total;
        *count = total;
        *done = 0u;
    }
}

// Ids of a write tile's selected positions from slot `first` on.  Thread t
// holds word t (positions tile0 + 32 t ..) and its exclusive count `ex` within
// the tile; the warp writes each of its 32 words' ids as one contiguous run
// (the position itself, or the list entry there).
template <bool kList>
__device__ __forceinline__ void where_emit(uint32_t word, uint32_t ex, uint32_t first, uint32_t tile0,
                                           const int32_t *__restrict__ in, int32_t *__restrict__ ids)
{
    const uint32_t lane = threadIdx.x & 31u, bit = 1u << lane, lt = bit - 1u;
    const uint32_t slot = first + ex;
    // word j of this warp covers positions pos + 32 j for this lane
    const uint32_t pos = tile0 + (threadIdx.x & ~31u) * 32u + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const uint32_t m = __shfl_sync(0xffffffffu, word, j);
        const uint32_t p = __shfl_sync(0xffffffffu, slot, j);
        if (m & bit) {
            const uint32_t q = pos + 32u * (uint32_t)j;
            ids[p + __popc(m & lt)] = kList ? in[q] : (int32_t)q;
        }
    }
}

template <bool kList>
__global__ void __launch_bounds__(kWhereNT) where_write_kernel(const uint32_t *__restrict__ bits,
                                                               const int32_t *__restrict__ off,
                                                               const int32_t *__restrict__ in,
                                                               int32_t *__restrict__ ids)
{
    __shared__ uint32_t s_warp[kWhereNT / 32 + 1];
    const uint32_t tile = blockIdx.x;
    const uint32_t word = bits[(size_t)tile * kWhereWords + threadIdx.x];
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<kWhereNT>(__popc(word), s_warp, &total);
    where_emit<kList>(word, ex, (uint32_t)off[tile], tile * kWhereTile, in, ids);
}

// At most one write tile of positions: both steps in one block.
template <int CMP, class T, bool kList>
__global__ void __launch_bounds__(kWhereNT) where_single_kernel(const T *__restrict__ c,
                                                                const int32_t *__restrict__ in, uint32_t n,
                                                                const uint32_t *__restrict__ n_dev, int64_t s,
                                                                int32_t *__restrict__ ids, uint32_t *__restrict__ count)
{
    __shared__ __align__(16) uint8_t s_map[kWhereWords * 4u];
    __shared__ uint32_t s_warp[kWhereNT / 32 + 1];
    const uint32_t tid = threadIdx.x;
    const uint32_t len = n_dev ? *n_dev : n;
    for (uint32_t b = tid; b < kWhereWords * 4u; b += kWhereNT)
        s_map[b] = (uint8_t)where_bits8<CMP, T, kList>(c, in, b * 8u, len, s);
    __syncthreads();
    const uint32_t word = reinterpret_cast<const uint32_t *>(s_map)[tid];
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<kWhereNT>(__popc(word), s_warp, &total);
    where_emit<kList>(word, ex, 0u, 0u, in, ids);
    if (tid == 0) *count = total;
}

// scatter_add with one value per listed id
__global__ void __launch_bounds__(256) view_add_values_i32_kernel(int32_t *__restrict__ c, const int32_t *__restrict__ ids,
                                                                  const uint32_t *__restrict__ count,
                                                                  const int32_t *__restrict__ vals, uint32_t n_vals,
                                                                  uint32_t *err)
{
    const uint32_t k = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && k > n_vals) atomicOr(err, ERR_RANGE);
    const uint32_t m = k < n_vals ? k : n_vals;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned int *>(c + ids[i]), (unsigned int)vals[i]);
}

__global__ void __launch_bounds__(256) view_add_values_u8_kernel(uint8_t *__restrict__ c, const int32_t *__restrict__ ids,
                                                                 const uint32_t *__restrict__ count,
                                                                 const int32_t *__restrict__ vals, uint32_t n_vals,
                                                                 uint32_t *err)
{
    const uint32_t k = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && k > n_vals) atomicOr(err, ERR_RANGE);
    const uint32_t m = k < n_vals ? k : n_vals;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const uint32_t id = (uint32_t)ids[i], sh = 8u * (id & 3u);
        const uint8_t add = (uint8_t)vals[i];
        uint32_t *word = reinterpret_cast<uint32_t *>(c + (id & ~3u));
        uint32_t old = *reinterpret_cast<volatile uint32_t *>(word);
        bool done = false;
        for (uint32_t attempt = 0; attempt < (1u << 24) && !done; ++attempt) {
            const uint32_t nv = (old & ~(0xFFu << sh)) | ((uint32_t)(uint8_t)((uint8_t)(old >> sh) + add) << sh);
            const uint32_t prev = atomicCAS(word, old, nv);
            done = (prev == old);
            old = prev;
        }
        if (!done) atomicOr(err, ERR_TIMEOUT);
    }
}

// ---------------------------------------------------------- view update ---
// Bounded compare-and-swap update of one word (lock-free: a failed attempt
// means another thread's update went in; the bound only guards against a
// hardware fault turning it into an endless loop).
template <class F>
__device__ __forceinline__ void cas_update(uint32_t *word, F f, uint32_t *err)
{
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(word);
    for (uint32_t attempt = 0; attempt < (1u << 24); ++attempt) {
        const uint32_t prev = atomicCAS(word, old, f(old));
        if (prev == old) return;
        old = prev;
    }
    atomicOr(err, ERR_TIMEOUT);
}

// Updates through a view: every thread takes kViewU listed ids per pass
// (list entries i0 + u kMapNT), so that their id loads, and then their column
// loads, are independent requests in flight together.  Ids of a filtered view
// are distinct, so all of a pass's reads can precede its writes; views that
// may repeat ids update through atomics.
constexpr int kViewU = 16;
constexpr uint32_t kNoId = 0xFFFFFFFFu;

__device__ __forceinline__ void load_ids(const int32_t *__restrict__ ids, uint32_t i0, uint32_t k, uint32_t id[kViewU])
{
#pragma unroll
    for (int u = 0; u < kViewU; ++u) {
        const uint32_t i = i0 + (uint32_t)u * kMapNT;
        id[u] = i < k ? (uint32_t)ids[i] : kNoId;
    }
}

template <int OP>
__device__ __forceinline__ void atomic_update_i32(int32_t *c, uint32_t id, int32_t s, uint32_t *err)
{
    if constexpr (OP == AMB_OP_ADD) {
        atomicAdd(reinterpret_cast<unsigned int *>(c + id), (unsigned int)s);
    } else if constexpr (OP == AMB_OP_SUB) {
        atomicSub(reinterpret_cast<unsigned int *>(c + id), (unsigned int)s);
    } else if constexpr (OP == AMB_OP_MIN) {
        atomicMin(c + id, s);
    } else if constexpr (OP == AMB_OP_MAX) {
        atomicMax(c + id, s);
    } else {
        cas_update(reinterpret_cast<uint32_t *>(c + id),
                   [s](uint32_t v) { return (uint32_t)apply_i32<OP>((int32_t)v, s); }, err);
    }
}

template <int OP, bool UNIQUE>
__global__ void __launch_bounds__(kMapNT) view_map_i32_kernel(int32_t *__restrict__ c, const int32_t *__restrict__ ids,
                                                              const uint32_t *__restrict__ count, int32_t s,
                                                              uint32_t *err)
{
    const uint32_t k = *count;
    for (uint32_t i0 = blockIdx.x * kMapNT * kViewU + threadIdx.x; i0 < k; i0 += gridDim.x * kMapNT * kViewU) {
        uint32_t id[kViewU];
        load_ids(ids, i0, k, id);
        if constexpr (UNIQUE || OP == AMB_OP_SET) {
            int32_t v[kViewU];
#pragma unroll
            for (int u = 0; u < kViewU; ++u)
                if (id[u] != kNoId) v[u] = c[id[u]];
#pragma unroll
            for (int u = 0; u < kViewU; ++u)
                if (id[u] != kNoId) c[id[u]] = apply_i32<OP>(v[u], s);
        } else {
#pragma unroll
            for (int u = 0; u < kViewU; ++u)
                if (id[u] != kNoId) atomic_update_i32<OP>(c, id[u], s, err);
        }
    }
}

template <int OP, bool UNIQUE>
__global__ void __launch_bounds__(kMapNT) view_map_u8_kernel(uint8_t *__restrict__ c, const int32_t *__restrict__ ids,
                                                             const uint32_t *__restrict__ count, uint8_t s,
                                                             uint32_t *err)
{
    const uint32_t k = *count;
    for (uint32_t i0 = blockIdx.x * kMapNT * kViewU + threadIdx.x; i0 < k; i0 += gridDim.x * kMapNT * kViewU) {
        uint32_t id[kViewU];
        load_ids(ids, i0, k, id);
        if constexpr (UNIQUE || OP == AMB_OP_SET) {
            uint8_t v[kViewU];
#pragma unroll
            for (int u = 0; u < kViewU; ++u)
                if (id[u] != kNoId) v[u] = c[id[u]];
#pragma unroll
            for (int u = 0; u < kViewU; ++u)
                if (id[u] != kNoId) c[id[u]] = apply_u8<OP>(v[u], s);
        } else {
#pragma unroll
            for (int u = 0; u < kViewU; ++u) {
                if (id[u] == kNoId) continue;
                // the byte's aligned 32-bit word (columns are padded to 4 bytes)
                const uint32_t sh = 8u * (id[u] & 3u);
                cas_update(reinterpret_cast<uint32_t *>(c + (id[u] & ~3u)),
                           [s, sh](uint32_t v) {
                               const uint8_t r = apply_u8<OP>((uint8_t)(v >> sh), s);
                               return (v & ~(0xFFu << sh)) | ((uint32_t)r << sh);
                           },
                           err);
            }
        }
    }
}

// random ids, one per listed id (counter-based: key (seed, rep), counter (id, step))
__global__ void __launch_bounds__(kMapNT) view_draw_kernel(const int32_t *__restrict__ ids,
                                                           const uint32_t *__restrict__ count,
                                                           int32_t *__restrict__ out, uint32_t *__restrict__ out_count,
                                                           uint32_t k0, uint32_t k1, uint32_t step, uint32_t word,
                                                           uint32_t range, int exclude_self)
{
    const uint32_t k = *count;
    if (blockIdx.x == 0 && threadIdx.x == 0) *out_count = k;
    const uint32_t m = exclude_self ? range - 1u : range;
    for (uint32_t i0 = blockIdx.x * kMapNT * kViewU + threadIdx.x; i0 < k; i0 += gridDim.x * kMapNT * kViewU) {
        uint32_t id[kViewU];
        load_ids(ids, i0, k, id);
#pragma unroll
        for (int u = 0; u < kViewU; ++u) {
            if (id[u] == kNoId) continue;
            const U4 q = philox(id[u], step, k0, k1);
            const uint32_t w = word == 0 ? q.w0 : word == 1 ? q.w1 : word == 2 ? q.w2 : q.w3;
            uint32_t r = below(w, m);
            if (exclude_self) r += (r >= id[u]) ? 1u : 0u;
            out[i0 + (uint32_t)u * kMapNT] = (int32_t)r;
        }
    }
}

// ids outside [0, n) in a caller-provided list
__global__ void ids_check_kernel(const int32_t *__restrict__ ids, uint32_t k, uint32_t n, uint32_t *err)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        if (ids[i] < 0 || (uint32_t)ids[i] >= n) atomicOr(err, ERR_RANGE);
}

__global__ void fill_kernel(uint8_t *__restrict__ p, size_t bytes, uint32_t word)
{
    uint32_t *w = reinterpret_cast<uint32_t *>(p);
    const size_t nw = bytes / 4u;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nw; i += (size_t)gridDim.x * blockDim.x) w[i] = word;
}

// ------------------------------------------------------- buffered writes ---
struct LogCols {
    void *ptr[kMaxLogCols];
    int32_t *win[kMaxLogCols];
    uint8_t dtype[kMaxLogCols];
};

__global__ void log_claim_kernel(const int32_t *__restrict__ ids, const int32_t *__restrict__ cols, uint32_t k,
                                 uint32_t base, LogCols lc)
{
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < k; e += gridDim.x * blockDim.x)
        atomicMax(&lc.win[cols[e]][ids[e]], (int32_t)(base + e));
}

__global__ void log_apply_kernel(const int32_t *__restrict__ ids, const int32_t *__restrict__ cols,
                                 const int64_t *__restrict__ vals, uint32_t k, uint32_t base, LogCols lc)
{
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < k; e += gridDim.x * blockDim.x) {
        const int32_t c = cols[e], id = ids[e];
        if (lc.win[c][id] != (int32_t)(base + e)) continue;  // a later record of this row wins
        if (lc.dtype[c] == AMB_DT_I32)
            static_cast<int32_t *>(lc.ptr[c])[id] = (int32_t)(uint32_t)(uint64_t)vals[e];
        else
            static_cast<uint8_t *>(lc.ptr[c])[id] = (uint8_t)(uint64_t)vals[e];
    }
}

__global__ void fill_i32_kernel(int32_t *__restrict__ p, uint32_t k, int32_t v)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) p[i] = v;
}

// ------------------------------------------------------------ grid walks ---
struct GridWalkArgs {
    int32_t *c[4];
    uint32_t size[4];
    uint32_t d, n, k0, k1, t0, steps;
    int moore, torus;
};

__device__ __forceinline__ int32_t wrap_coord(int32_t v, int32_t o, uint32_t size)
{
    int64_t s = (int64_t)v + o;
    if (s < 0) s += size;
    if (s >= (int64_t)size) s -= size;
    return (int32_t)s;
}

// m -> (m / v, m % v) for a per-dimension neighbour count v in {1, 2, 3}
__device__ __forceinline__ uint32_t divmod123(uint32_t &m, uint32_t v)
{
    const uint32_t q3 = m / 3u, q2 = m >> 1;
    const uint32_t r = v == 3u ? m - 3u * q3 : v == 2u ? (m & 1u) : 0u;
    m = v == 3u ? q3 : v == 2u ? q2 : m;
    return r;
}

// Dimension count and neighbourhood are template arguments, so the
// per-dimension loops unroll and a torus divides by the constant 3.
template <uint32_t D, bool MOORE, bool TORUS>
__global__ void __launch_bounds__(256) grid_walk_kernel(GridWalkArgs a, uint32_t *err)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        int32_t c[D];
        bool ok = true;
#pragma unroll
        for (uint32_t q = 0; q < D; ++q) {
            c[q] = a.c[q][i];
            ok &= c[q] >= 0 && (uint32_t)c[q] < a.size[q];
        }
        if (!ok) {
            atomicOr(err, ERR_RANGE);
            continue;
        }
        for (uint32_t j = 0; j < a.steps; ++j) {
            const U4 u = philox(i, a.t0 + j, a.k0, a.k1);
            int32_t off[D];
#pragma unroll
            for (uint32_t q = 0; q < D; ++q) off[q] = 0;
            if constexpr (MOORE) {
                // per dimension the admissible offsets (-1 if inside, 0, +1 if
                // inside), in order; m enumerates their product, the all-zero
                // offset left out
                uint32_t v[D], lo[D], total = 1, center = 0;
#pragma unroll
                for (uint32_t q = 0; q < D; ++q) {
                    const bool dn = TORUS || c[q] > 0, up = TORUS || (uint32_t)c[q] + 1u < a.size[q];
                    lo[q] = dn ? 1u : 0u;  // index of the zero offset in this dimension's list
                    v[q] = 1u + (dn ? 1u : 0u) + (up ? 1u : 0u);
                    center += lo[q] * total;
                    total *= v[q];
                }
                const uint32_t cnt = total - 1u;
                if (cnt == 0) continue;
                uint32_t m = below(u.w0, cnt);
                if (m >= center) ++m;  // skip the zero offset
#pragma unroll
                for (uint32_t q = 0; q < D; ++q) {
                    const uint32_t r = TORUS ? m % 3u : divmod123(m, v[q]);
                    if (TORUS) m /= 3u;
                    off[q] = (int32_t)r - (int32_t)lo[q];
                }
            } else {
                // von Neumann: the admissible unit moves, dimension by
                // dimension, -1 before +1
                uint32_t cnt = 0;
#pragma unroll
                for (uint32_t q = 0; q < D; ++q) {
                    cnt += (TORUS || c[q] > 0) ? 1u : 0u;
                    cnt += (TORUS || (uint32_t)c[q] + 1u < a.size[q]) ? 1u : 0u;
                }
                if (cnt == 0) continue;
                uint32_t m = below(u.w0, cnt);
                bool done = false;
#pragma unroll
                for (uint32_t q = 0; q < D; ++q) {
                    if (!done && (TORUS || c[q] > 0)) {
                        if (m == 0) {
                            off[q] = -1;
                            done = true;
                        } else {
                            --m;
                        }
                    }
                    if (!done && (TORUS || (uint32_t)c[q] + 1u < a.size[q])) {
                        if (m == 0) {
                            off[q] = 1;
                            done = true;
                        } else {
                            --m;
                        }
                    }
                }
            }
#pragma unroll
            for (uint32_t q = 0; q < D; ++q) c[q] = wrap_coord(c[q], off[q], a.size[q]);
        }
#pragma unroll
        for (uint32_t q = 0; q < D; ++q) a.c[q][i] = c[q];
    }
}

unsigned map_grid(uint64_t work)
{
    return grid_for(work, kMapNT, 16u);
}

// ----------------------------------------------------------- dispatch ---
amb_status bad_op(int op) { return fail(AMB_EINVAL, "unknown operation %d", op); }

amb_status launch_map(const Column &col, uint32_t n, int op, int64_t s, cudaStream_t st)
{
    if (n == 0) return AMB_OK;
    if (col.dtype == AMB_DT_I32) {
        int32_t *c = static_cast<int32_t *>(col.ptr);
        const int32_t v = (int32_t)(uint32_t)s;
        const unsigned g = map_grid(n / 4u + 1u);
        switch (op) {
        case AMB_OP_SET: map_i32_kernel<AMB_OP_SET><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_ADD: map_i32_kernel<AMB_OP_ADD><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_SUB: map_i32_kernel<AMB_OP_SUB><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_MUL: map_i32_kernel<AMB_OP_MUL><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_MIN: map_i32_kernel<AMB_OP_MIN><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_MAX: map_i32_kernel<AMB_OP_MAX><<<g, kMapNT, 0, st>>>(c, n, v); break;
        default: return bad_op(op);
        }
    } else {
        uint8_t *c = static_cast<uint8_t *>(col.ptr);
        const uint8_t v = (uint8_t)s;
        const unsigned g = map_grid(n / 16u + 1u);
        switch (op) {
        case AMB_OP_SET: map_u8_kernel<AMB_OP_SET><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_ADD: map_u8_kernel<AMB_OP_ADD><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_SUB: map_u8_kernel<AMB_OP_SUB><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_MUL: map_u8_kernel<AMB_OP_MUL><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_MIN: map_u8_kernel<AMB_OP_MIN><<<g, kMapNT, 0, st>>>(c, n, v); break;
        case AMB_OP_MAX: map_u8_kernel<AMB_OP_MAX><<<g, kMapNT, 0, st>>>(c, n, v); break;
        default: return bad_op(op);
        }
    }
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

template <class D, class S>
amb_status launch_map_col_t(D *d, const S *src, uint32_t n, int op, cudaStream_t st)
{
    const unsigned g = map_grid(n);
    switch (op) {
    case AMB_OP_SET: map_col_kernel<AMB_OP_SET><<<g, kMapNT, 0, st>>>(d, src, n); break;
    case AMB_OP_ADD: map_col_kernel<AMB_OP_ADD><<<g, kMapNT, 0, st>>>(d, src, n); break;
    case AMB_OP_SUB: map_col_kernel<AMB_OP_SUB><<<g, kMapNT, 0, st>>>(d, src, n); break;
    case AMB_OP_MUL: map_col_kernel<AMB_OP_MUL><<<g, kMapNT, 0, st>>>(d, src, n); break;
    case AMB_OP_MIN: map_col_kernel<AMB_OP_MIN><<<g, kMapNT, 0, st>>>(d, src, n); break;
    case AMB_OP_MAX: map_col_kernel<AMB_OP_MAX><<<g, kMapNT, 0, st>>>(d, src, n); break;
    default: return bad_op(op);
    }
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

// Scratch of where(): predicate words, per-tile counts and their scan for up
// to `tiles` write tiles (grown on demand: a view's list may be longer than
// the table).  Frees are stream-ordered, after any launch still using them.
amb_status ensure_where_scratch(amb_table *t, uint32_t tiles, cudaStream_t st)
{
    if (!t->where_done) {
        AMB_TRY(dalloc(&t->where_done, 1, st));
        AMB_TRY_CUDA(cudaMemsetAsync(t->where_done, 0, sizeof(uint32_t), st));
    }
    if (tiles <= t->where_tiles) return AMB_OK;
    dfree(t->where_bits, st);
    dfree(t->where_cnt, st);
    dfree(t->where_off, st);
    t->where_tiles = 0;
    AMB_TRY(dalloc(&t->where_bits, (size_t)tiles * kWhereWords, st));
    AMB_TRY(dalloc(&t->where_cnt, tiles, st));
    AMB_TRY(dalloc(&t->where_off, (size_t)tiles + 1u, st));
    t->where_tiles = tiles;
    return AMB_OK;
}

// where over positions 0 .. n-1 of the column's rows (kList false) or of the
// view list `in` (kList true; n_dev holds its length, at most n); the
// selected ids, in position order, go to `out`.
template <class T, bool kList>
amb_status launch_where_t(amb_table *t, const T *c, const int32_t *in, uint32_t n, const uint32_t *n_dev, int cmp,
                          int64_t s, amb_view *out)
{
    cudaStream_t st = t->stream;
    if (n == 0) {
        AMB_TRY_CUDA(cudaMemsetAsync(out->count, 0, sizeof(uint32_t), st));
        return AMB_OK;
    }
    using Sp = WhereSpan<T, kList>;
    const uint32_t n_tiles = (uint32_t)(((uint64_t)n + kWhereTile - 1u) / kWhereTile);
    const uint32_t n_spans = (uint32_t)(((uint64_t)n + Sp::kItems - 1u) / Sp::kItems);
    if (n_tiles > 1u) AMB_TRY(ensure_where_scratch(t, n_tiles, st));
#define WHERE_CASE(C)                                                                                            \
    case C:                                                                                                      \
        if (n_tiles == 1u) {                                                                                     \
            where_single_kernel<C, T, kList><<<1, kWhereNT, 0, st>>>(c, in, n, n_dev, s, out->ids, out->count);  \
        } else {                                                                                                 \
            where_flags_kernel<C, T, kList><<<n_spans, kWhereNT, 0, st>>>(c, in, n, n_dev, s, t->where_bits,     \
                                                                          t->where_cnt, t->where_off, n_tiles,  \
                                                                          t->where_done, out->count);           \
            AMB_TRY_CUDA(cudaGetLastError());                                                                    \
            where_write_kernel<kList><<<n_tiles, kWhereNT, 0, st>>>(t->where_bits, t->where_off, in, out->ids); \
        }                                                                                                        \
        break;
    switch (cmp) {
        WHERE_CASE(AMB_CMP_EQ)
        WHERE_CASE(AMB_CMP_NE)
        WHERE_CASE(AMB_CMP_LT)
        WHERE_CASE(AMB_CMP_LE)
        WHERE_CASE(AMB_CMP_GT)
        WHERE_CASE(AMB_CMP_GE)
    default: return fail(AMB_EINVAL, "unknown comparison %d", cmp);
    }
#undef WHERE_CASE
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

template <bool UNIQUE>
amb_status launch_view_map_t(amb_view *v, const Column &col, int op, int64_t s)
{
    amb_table *t = v->t;
    cudaStream_t st = t->stream;
    if (v->capacity == 0) return AMB_OK;
    const unsigned g = map_grid(((uint64_t)v->capacity + kViewU - 1u) / kViewU);
#define VM_CASE(K, O, val) \
    case O: K<O, UNIQUE><<<g, kMapNT, 0, st>>>(c, v->ids, v->count, val, t->err); break;
    if (col.dtype == AMB_DT_I32) {
        int32_t *c = static_cast<int32_t *>(col.ptr);
        const int32_t val = (int32_t)(uint32_t)s;
        switch (op) {
            VM_CASE(view_map_i32_kernel, AMB_OP_SET, val)
            VM_CASE(view_map_i32_kernel, AMB_OP_ADD, val)
            VM_CASE(view_map_i32_kernel, AMB_OP_SUB, val)
            VM_CASE(view_map_i32_kernel, AMB_OP_MUL, val)
            VM_CASE(view_map_i32_kernel, AMB_OP_MIN, val)
            VM_CASE(view_map_i32_kernel, AMB_OP_MAX, val)
        default: return bad_op(op);
        }
    } else {
        uint8_t *c = static_cast<uint8_t *>(col.ptr);
        const uint8_t val = (uint8_t)s;
        switch (op) {
            VM_CASE(view_map_u8_kernel, AMB_OP_SET, val)
            VM_CASE(view_map_u8_kernel, AMB_OP_ADD, val)
            VM_CASE(view_map_u8_kernel, AMB_OP_SUB, val)
            VM_CASE(view_map_u8_kernel, AMB_OP_MUL, val)
            VM_CASE(view_map_u8_kernel, AMB_OP_MIN, val)
            VM_CASE(view_map_u8_kernel, AMB_OP_MAX, val)
        default: return bad_op(op);
        }
    }
#undef VM_CASE
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status table_error(amb_table *t)
{
    uint32_t h = 0;
    AMB_TRY_CUDA(cudaMemcpyAsync(&h, t->err, sizeof(h), cudaMemcpyDeviceToHost, t->stream));
    AMB_TRY_CUDA(cudaStreamSynchronize(t->stream));
    if (h & ERR_TIMEOUT) return fail(AMB_ETIMEOUT, "a bounded device-side wait ran out (error word 0x%x)", h);
    if (h & ERR_RANGE) {
        // caller input (ids, coordinates) out of range: reported once, the table stays usable
        AMB_TRY_CUDA(cudaMemsetAsync(t->err, 0, sizeof(uint32_t), t->stream));
        AMB_TRY_CUDA(cudaStreamSynchronize(t->stream));
        return fail(AMB_EINVAL, "an id or coordinate outside its range was given (error word 0x%x)", h);
    }
    if (h) return fail(AMB_EINVARIANT, "device error word 0x%x", h);
    return AMB_OK;
}

amb_status get_col(amb_table *t, int col, Column **out)
{
    if (!t) return fail(AMB_EINVAL, "null table");
    if (col < 0 || (size_t)col >= t->cols.size()) return fail(AMB_EINVAL, "unknown column %d", col);
    *out = &t->cols[(size_t)col];
    return AMB_OK;
}

size_t col_bytes(amb_dtype dt, uint32_t n)
{
    return dt == AMB_DT_I32 ? (size_t)n * 4u : (((size_t)n + 3u) & ~(size_t)3u);
}

amb_status new_view(amb_table *t, uint32_t capacity, bool unique, amb_view **out)
{
    amb_view *v = new (std::nothrow) amb_view();
    if (!v) return fail(AMB_ENOMEM, "host allocation failed");
    v->t = t;
    v->capacity = capacity;
    v->unique = unique;
    amb_status st = dalloc(&v->ids, capacity, t->stream);
    if (st == AMB_OK) st = dalloc(&v->count, 1, t->stream);
    if (st != AMB_OK) {
        dfree(v->ids, t->stream);
        dfree(v->count, t->stream);
        delete v;
        return st;
    }
    t->live_views += 1;
    *out = v;
    return AMB_OK;
}

}  // namespace

extern "C" {

amb_status amb_table_create(uint32_t n, void *cuda_stream, amb_table **out)
{
    if (!out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    if (n > 0x7FFFFFFFu) return fail(AMB_EINVAL, "n must be < 2^31");
    amb_table *t = new (std::nothrow) amb_table();
    if (!t) return fail(AMB_ENOMEM, "host allocation failed");
    t->n = n;
    t->stream = (cudaStream_t)cuda_stream;
    amb_status st = dalloc(&t->err, 1, t->stream);
    if (st == AMB_OK && cudaMemsetAsync(t->err, 0, sizeof(uint32_t), t->stream) != cudaSuccess)
        st = fail(AMB_ECUDA, "memset failed");
    if (st != AMB_OK) {
        dfree(t->err, t->stream);
        delete t;
        return st;
    }
    *out = t;
    return AMB_OK;
}

amb_status amb_table_destroy(amb_table *t)
{
    if (!t) return AMB_OK;
    if (t->live_views) return fail(AMB_EBUSY, "%d views of this table are still alive", t->live_views);
    for (Column &c : t->cols) dfree(c.ptr, t->stream);
    dfree(t->err, t->stream);
    dfree(t->where_bits, t->stream);
    dfree(t->where_cnt, t->stream);
    dfree(t->where_off, t->stream);
    dfree(t->where_done, t->stream);
    cudaStreamSynchronize(t->stream);
    delete t;
    return AMB_OK;
}

amb_status amb_table_add_column(amb_table *t, const char *name, amb_dtype dtype, int64_t fill, int *col_out)
{
    if (!t || !name || !col_out) return fail(AMB_EINVAL, "null pointer");
    if (dtype != AMB_DT_I32 && dtype != AMB_DT_U8) return fail(AMB_EINVAL, "unknown dtype %d", (int)dtype);
    if (!*name) return fail(AMB_EINVAL, "empty column name");
    for (const Column &c : t->cols)
        if (c.name == name) return fail(AMB_EINVAL, "column '%s' exists", name);
    Column c;
    c.name = name;
    c.dtype = dtype;
    const size_t bytes = col_bytes(dtype, t->n);
    unsigned char *p = nullptr;
    AMB_TRY(dalloc(&p, bytes, t->stream));
    c.ptr = p;
    uint32_t word;
    if (dtype == AMB_DT_I32) {
        word = (uint32_t)fill;
    } else {
        const uint32_t b = (uint8_t)fill;
        word = b | (b << 8) | (b << 16) | (b << 24);
    }
    if (bytes) {
        fill_kernel<<<grid_for(bytes / 4u, 256, 8u), 256, 0, t->stream>>>(p, bytes, word);
        if (cudaGetLastError() != cudaSuccess) {
            dfree(c.ptr, t->stream);
            return fail(AMB_ECUDA, "fill launch failed");
        }
    }
    try {
        t->cols.push_back(c);
    } catch (...) {
        dfree(c.ptr, t->stream);
        return fail(AMB_ENOMEM, "host allocation failed");
    }
    *col_out = (int)t->cols.size() - 1;
    return AMB_OK;
}

amb_status amb_table_find_column(amb_table *t, const char *name, int *col_out)
{
    if (!t || !name || !col_out) return fail(AMB_EINVAL, "null pointer");
    for (size_t i = 0; i < t->cols.size(); ++i)
        if (t->cols[i].name == name) {
            *col_out = (int)i;
            return AMB_OK;
        }
    return fail(AMB_ENOTFOUND, "no column '%s'", name);
}

amb_status amb_table_rows(amb_table *t, uint32_t *n)
{
    if (!t || !n) return fail(AMB_EINVAL, "null pointer");
    *n = t->n;
    return AMB_OK;
}

amb_status amb_table_write(amb_table *t, int col, const void *src, size_t n, int src_on_device)
{
    AMB_TRACE("amb_table_write");
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    if (n != t->n) return fail(AMB_EINVAL, "column length %zu != n = %u", n, t->n);
    if (!src && n) return fail(AMB_EINVAL, "null pointer");
    const size_t bytes = (c->dtype == AMB_DT_I32 ? 4u : 1u) * n;
    if (bytes)
        AMB_TRY_CUDA(cudaMemcpyAsync(c->ptr, src, bytes, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     t->stream));
    if (!src_on_device) AMB_TRY_CUDA(cudaStreamSynchronize(t->stream));  // the caller may reuse src
    return AMB_OK;
}

amb_status amb_table_read(amb_table *t, int col, void *dst, size_t n, int dst_on_device)
{
    AMB_TRACE("amb_table_read");
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    if (n != t->n) return fail(AMB_EINVAL, "column length %zu != n = %u", n, t->n);
    if (!dst && n) return fail(AMB_EINVAL, "null pointer");
    AMB_TRY(table_error(t));
    const size_t bytes = (c->dtype == AMB_DT_I32 ? 4u : 1u) * n;
    if (bytes)
        AMB_TRY_CUDA(cudaMemcpyAsync(dst, c->ptr, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     t->stream));
    AMB_TRY_CUDA(cudaStreamSynchronize(t->stream));
    return AMB_OK;
}

amb_status amb_table_map(amb_table *t, int col, amb_op op, int64_t scalar)
{
    AMB_TRACE("amb_table_map");
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    return launch_map(*c, t->n, op, scalar, t->stream);
}

amb_status amb_table_map_col(amb_table *t, int dst, amb_op op, int src)
{
    AMB_TRACE("amb_table_map_col");
    Column *d = nullptr, *s = nullptr;
    AMB_TRY(get_col(t, dst, &d));
    AMB_TRY(get_col(t, src, &s));
    if (t->n == 0) return AMB_OK;
    if (d->dtype == AMB_DT_I32 && s->dtype == AMB_DT_I32)
        return launch_map_col_t(static_cast<int32_t *>(d->ptr), static_cast<const int32_t *>(s->ptr), t->n, op, t->stream);
    if (d->dtype == AMB_DT_I32)
        return launch_map_col_t(static_cast<int32_t *>(d->ptr), static_cast<const uint8_t *>(s->ptr), t->n, op, t->stream);
    if (s->dtype == AMB_DT_I32)
        return launch_map_col_t(static_cast<uint8_t *>(d->ptr), static_cast<const int32_t *>(s->ptr), t->n, op, t->stream);
    return launch_map_col_t(static_cast<uint8_t *>(d->ptr), static_cast<const uint8_t *>(s->ptr), t->n, op, t->stream);
}

amb_status amb_table_where(amb_table *t, int col, amb_cmp cmp, int64_t scalar, amb_view **out)
{
    AMB_TRACE("amb_table_where");
    if (!out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    if ((int)cmp < 0 || (int)cmp > AMB_CMP_GE) return fail(AMB_EINVAL, "unknown comparison %d", (int)cmp);
    amb_view *v = nullptr;
    AMB_TRY(new_view(t, t->n, true, &v));
    const amb_status st = c->dtype == AMB_DT_I32
                              ? launch_where_t<int32_t, false>(t, static_cast<const int32_t *>(c->ptr), nullptr, t->n,
                                                               nullptr, cmp, scalar, v)
                              : launch_where_t<uint8_t, false>(t, static_cast<const uint8_t *>(c->ptr), nullptr, t->n,
                                                               nullptr, cmp, scalar, v);
    if (st != AMB_OK) {
        amb_view_destroy(v);
        return st;
    }
    *out = v;
    return AMB_OK;
}

amb_status amb_view_from_ids(amb_table *t, const int32_t *ids, size_t k, int ids_on_device, amb_view **out)
{
    AMB_TRACE("amb_view_from_ids");
    if (!t || !out || (!ids && k)) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    if (k > 0x7FFFFFFFu) return fail(AMB_EINVAL, "too many ids");
    if (!ids_on_device)
        for (size_t i = 0; i < k; ++i)
            if (ids[i] < 0 || (uint32_t)ids[i] >= t->n) return fail(AMB_EINVAL, "id %d at %zu outside [0, %u)", ids[i], i, t->n);
    amb_view *v = nullptr;
    AMB_TRY(new_view(t, (uint32_t)k, false, &v));
    const uint32_t kk = (uint32_t)k;
    amb_status st = AMB_OK;
    if (k && cudaMemcpyAsync(v->ids, ids, k * sizeof(int32_t), ids_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             t->stream) != cudaSuccess)
        st = fail(AMB_ECUDA, "id copy failed");
    if (st == AMB_OK && cudaMemcpyAsync(v->count, &kk, sizeof(kk), cudaMemcpyHostToDevice, t->stream) != cudaSuccess)
        st = fail(AMB_ECUDA, "count copy failed");
    if (st == AMB_OK && ids_on_device && k) {
        ids_check_kernel<<<grid_for(k, 256, 8u), 256, 0, t->stream>>>(v->ids, kk, t->n, t->err);
        if (cudaGetLastError() != cudaSuccess) st = fail(AMB_ECUDA, "check launch failed");
    }
    if (st == AMB_OK) st = table_error(t);  // also: the host copies are complete
    if (st != AMB_OK) {
        // a range error stays recorded in the table's error word
        amb_view_destroy(v);
        return st;
    }
    *out = v;
    return AMB_OK;
}

amb_status amb_view_draw(amb_view *v, uint64_t seed, uint32_t replicate, uint32_t step, uint32_t word, uint32_t range,
                         int exclude_self, amb_view **out)
{
    AMB_TRACE("amb_view_draw");
    if (!v || !out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    if (seed > 0xFFFFFFFFull) return fail(AMB_EINVAL, "seed must be < 2^32");
    if (word > 3) return fail(AMB_EINVAL, "word must be 0..3");
    amb_table *t = v->t;
    // the drawn ids address rows of the table, so the range is at most n
    if (range > t->n || range < (exclude_self ? 2u : 1u))
        return fail(AMB_EINVAL, "range %u out of bounds (at most the table's %u rows; exclude_self needs >= 2)", range,
                    t->n);
    amb_view *r = nullptr;
    AMB_TRY(new_view(t, v->capacity, false, &r));
    if (v->capacity) {
        view_draw_kernel<<<map_grid(((uint64_t)v->capacity + kViewU - 1u) / kViewU), kMapNT, 0, t->stream>>>(v->ids, v->count, r->ids, r->count, (uint32_t)seed,
                                                                          replicate, step, word, range, exclude_self);
    } else {
        cudaMemsetAsync(r->count, 0, sizeof(uint32_t), t->stream);
    }
    if (cudaGetLastError() != cudaSuccess) {
        amb_view_destroy(r);
        return fail(AMB_ECUDA, "draw launch failed");
    }
    *out = r;
    return AMB_OK;
}

amb_status amb_view_where(amb_view *v, int col, amb_cmp cmp, int64_t scalar, amb_view **out)
{
    AMB_TRACE("amb_view_where");
    if (!v || !out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    amb_table *t = v->t;
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    if ((int)cmp < 0 || (int)cmp > AMB_CMP_GE) return fail(AMB_EINVAL, "unknown comparison %d", (int)cmp);
    amb_view *r = nullptr;
    AMB_TRY(new_view(t, v->capacity, v->unique, &r));
    const amb_status res =
        c->dtype == AMB_DT_I32
            ? launch_where_t<int32_t, true>(t, static_cast<const int32_t *>(c->ptr), v->ids, v->capacity, v->count,
                                            cmp, scalar, r)
            : launch_where_t<uint8_t, true>(t, static_cast<const uint8_t *>(c->ptr), v->ids, v->capacity, v->count,
                                            cmp, scalar, r);
    if (res != AMB_OK) {
        amb_view_destroy(r);
        return res;
    }
    *out = r;
    return AMB_OK;
}

amb_status amb_view_scatter_add_values(amb_view *v, int col, const int32_t *values, size_t n_values)
{
    AMB_TRACE("amb_view_scatter_add_values");
    if (!v || (!values && n_values)) return fail(AMB_EINVAL, "null pointer");
    amb_table *t = v->t;
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    if (n_values > 0xFFFFFFFFu) return fail(AMB_EINVAL, "too many values");
    if (v->capacity == 0) return AMB_OK;
    const unsigned g = map_grid(v->capacity);
    if (c->dtype == AMB_DT_I32)
        view_add_values_i32_kernel<<<g, 256, 0, t->stream>>>(static_cast<int32_t *>(c->ptr), v->ids, v->count, values,
                                                             (uint32_t)n_values, t->err);
    else
        view_add_values_u8_kernel<<<g, 256, 0, t->stream>>>(static_cast<uint8_t *>(c->ptr), v->ids, v->count, values,
                                                            (uint32_t)n_values, t->err);
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

amb_status amb_view_map(amb_view *v, int col, amb_op op, int64_t scalar)
{
    AMB_TRACE("amb_view_map");
    if (!v) return fail(AMB_EINVAL, "null view");
    Column *c = nullptr;
    AMB_TRY(get_col(v->t, col, &c));
    return v->unique ? launch_view_map_t<true>(v, *c, op, scalar) : launch_view_map_t<false>(v, *c, op, scalar);
}

amb_status amb_view_scatter_add(amb_view *v, int col, int64_t value)
{
    return amb_view_map(v, col, AMB_OP_ADD, value);
}

amb_status amb_view_count(amb_view *v, size_t *count)
{
    if (!v || !count) return fail(AMB_EINVAL, "null pointer");
    uint32_t h = 0;
    AMB_TRY_CUDA(cudaMemcpyAsync(&h, v->count, sizeof(h), cudaMemcpyDeviceToHost, v->t->stream));
    AMB_TRY(table_error(v->t));
    *count = h;
    return AMB_OK;
}

amb_status amb_view_ids(amb_view *v, int32_t *dst, size_t cap, int dst_on_device, size_t *count)
{
    AMB_TRACE("amb_view_ids");
    if (!v || (!dst && cap)) return fail(AMB_EINVAL, "null pointer");
    size_t k = 0;
    AMB_TRY(amb_view_count(v, &k));
    if (count) *count = k;
    const size_t m = std::min(k, cap);
    if (m)
        AMB_TRY_CUDA(cudaMemcpyAsync(dst, v->ids, m * sizeof(int32_t),
                                     dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, v->t->stream));
    AMB_TRY_CUDA(cudaStreamSynchronize(v->t->stream));
    return AMB_OK;
}

amb_status amb_view_destroy(amb_view *v)
{
    if (!v) return AMB_OK;
    dfree(v->ids, v->t->stream);
    dfree(v->count, v->t->stream);
    v->t->live_views -= 1;
    delete v;
    return AMB_OK;
}

amb_status amb_table_synchronize(amb_table *t)
{
    if (!t) return fail(AMB_EINVAL, "null table");
    return table_error(t);
}

amb_status amb_log_create(amb_table *t, uint32_t capacity, amb_log **out)
{
    if (!t || !out) return fail(AMB_EINVAL, "null pointer");
    *out = nullptr;
    if (capacity > 0x7FFFFFFFu) return fail(AMB_EINVAL, "capacity must be < 2^31");
    amb_log *l = new (std::nothrow) amb_log();
    if (!l) return fail(AMB_ENOMEM, "host allocation failed");
    l->t = t;
    l->capacity = capacity;
    amb_status st = dalloc(&l->ids, capacity, t->stream);
    if (st == AMB_OK) st = dalloc(&l->cols, capacity, t->stream);
    if (st == AMB_OK) st = dalloc(&l->vals, capacity, t->stream);
    if (st != AMB_OK) {
        dfree(l->ids, t->stream);
        dfree(l->cols, t->stream);
        dfree(l->vals, t->stream);
        delete l;
        return st;
    }
    t->live_views += 1;
    *out = l;
    return AMB_OK;
}

amb_status amb_log_record(amb_log *l, int col, const int32_t *ids, const int64_t *values, size_t k, int on_device)
{
    if (!l || ((!ids || !values) && k)) return fail(AMB_EINVAL, "null pointer");
    amb_table *t = l->t;
    Column *c = nullptr;
    AMB_TRY(get_col(t, col, &c));
    if (col >= kMaxLogCols) return fail(AMB_EINVAL, "a log addresses the first %d columns only", kMaxLogCols);
    if (k > (size_t)(l->capacity - l->count)) return fail(AMB_EINVAL, "log full (%u of %u records)", l->count, l->capacity);
    if (k == 0) return AMB_OK;
    if (!on_device)
        for (size_t i = 0; i < k; ++i)
            if (ids[i] < 0 || (uint32_t)ids[i] >= t->n) return fail(AMB_EINVAL, "id %d at %zu outside [0, %u)", ids[i], i, t->n);
    cudaStream_t s = t->stream;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    AMB_TRY_CUDA(cudaMemcpyAsync(l->ids + l->count, ids, k * sizeof(int32_t), kind, s));
    AMB_TRY_CUDA(cudaMemcpyAsync(l->vals + l->count, values, k * sizeof(int64_t), kind, s));
    fill_i32_kernel<<<grid_for(k, 256, 8u), 256, 0, s>>>(l->cols + l->count, (uint32_t)k, col);
    AMB_TRY_CUDA(cudaGetLastError());
    if (on_device) {
        ids_check_kernel<<<grid_for(k, 256, 8u), 256, 0, s>>>(l->ids + l->count, (uint32_t)k, t->n, t->err);
        AMB_TRY_CUDA(cudaGetLastError());
        AMB_TRY(table_error(t));  // a bad id leaves the log unchanged (count not advanced)
    } else {
        AMB_TRY_CUDA(cudaStreamSynchronize(s));  // the caller may reuse its buffers
    }
    if (l->used.size() < t->cols.size()) l->used.resize(t->cols.size(), false);
    l->used[(size_t)col] = true;
    l->count += (uint32_t)k;
    return AMB_OK;
}

amb_status amb_log_pending(amb_log *l, size_t *k)
{
    if (!l || !k) return fail(AMB_EINVAL, "null pointer");
    *k = l->count;
    return AMB_OK;
}

amb_status amb_log_flush(amb_log *l)
{
    AMB_TRACE("amb_log_flush");
    if (!l) return fail(AMB_EINVAL, "null log");
    amb_table *t = l->t;
    cudaStream_t s = t->stream;
    if (l->count == 0) return AMB_OK;
    if (l->win.size() < t->cols.size()) l->win.resize(t->cols.size(), nullptr);
    // record numbers stay below 2^31: start again from 0 with cleared words
    // when this flush would pass that
    if ((uint64_t)l->base + l->count >= 0x7FFFFFFFull) {
        for (int32_t *w : l->win)
            if (w) AMB_TRY_CUDA(cudaMemsetAsync(w, 0xFF, (size_t)t->n * sizeof(int32_t), s));
        l->base = 0;
    }
    LogCols lc;
    memset(&lc, 0, sizeof(lc));
    for (size_t c = 0; c < t->cols.size() && c < (size_t)kMaxLogCols; ++c) {
        lc.ptr[c] = t->cols[c].ptr;
        lc.dtype[c] = (uint8_t)t->cols[c].dtype;
        if (c < l->used.size() && l->used[c] && !l->win[c]) {
            AMB_TRY(dalloc(&l->win[c], t->n, s));
            AMB_TRY_CUDA(cudaMemsetAsync(l->win[c], 0xFF, (size_t)t->n * sizeof(int32_t), s));  // -1
        }
        lc.win[c] = l->win[c];
    }
    const unsigned g = grid_for(l->count, 256, 16u);
    log_claim_kernel<<<g, 256, 0, s>>>(l->ids, l->cols, l->count, l->base, lc);
    log_apply_kernel<<<g, 256, 0, s>>>(l->ids, l->cols, l->vals, l->count, l->base, lc);
    AMB_TRY_CUDA(cudaGetLastError());
    l->base += l->count;
    l->count = 0;
    std::fill(l->used.begin(), l->used.end(), false);
    return AMB_OK;
}

amb_status amb_debug_log_base(amb_log *l, uint32_t base)
{
    if (!l) return fail(AMB_EINVAL, "null log");
    if (l->count) return fail(AMB_EINVAL, "records are pending");
    if (base >= 0x80000000u) return fail(AMB_EINVAL, "base must be < 2^31");
    l->base = base;
    return AMB_OK;
}

amb_status amb_log_destroy(amb_log *l)
{
    if (!l) return AMB_OK;
    cudaStream_t s = l->t->stream;
    dfree(l->ids, s);
    dfree(l->cols, s);
    dfree(l->vals, s);
    for (int32_t *w : l->win) dfree(w, s);
    l->t->live_views -= 1;
    delete l;
    return AMB_OK;
}

amb_status amb_table_grid_walk(amb_table *t, const int *cols, uint32_t d, const uint32_t *sizes, int moore, int torus,
                               uint64_t seed, uint32_t replicate, uint32_t step, uint32_t steps)
{
    AMB_TRACE("amb_table_grid_walk");
    if (!t || !cols || !sizes) return fail(AMB_EINVAL, "null pointer");
    if (d < 1 || d > 4) return fail(AMB_EINVAL, "grids have 1 to 4 dimensions");
    if (seed > 0xFFFFFFFFull) return fail(AMB_EINVAL, "seed must be < 2^32");
    if ((uint64_t)step + steps >= 0xFFFFFFFFull) return fail(AMB_EINVAL, "step index would reach 2^32 - 1");
    GridWalkArgs a;
    memset(&a, 0, sizeof(a));
    for (uint32_t q = 0; q < d; ++q) {
        Column *c = nullptr;
        AMB_TRY(get_col(t, cols[q], &c));
        if (c->dtype != AMB_DT_I32) return fail(AMB_EINVAL, "grid coordinates are int32 columns");
        if (sizes[q] < 1 || sizes[q] > 0x7FFFFFFFu) return fail(AMB_EINVAL, "grid sizes must be in [1, 2^31)");
        for (uint32_t r = 0; r < q; ++r)
            if (cols[r] == cols[q]) return fail(AMB_EINVAL, "a column appears twice");
        a.c[q] = static_cast<int32_t *>(c->ptr);
        a.size[q] = sizes[q];
    }
    if (t->n == 0 || steps == 0) return AMB_OK;
    a.d = d;
    a.n = t->n;
    a.k0 = (uint32_t)seed;
    a.k1 = replicate;
    a.t0 = step;
    a.steps = steps;
    a.moore = moore != 0;
    a.torus = torus != 0;
    const unsigned g = grid_for(t->n, 256, 32u);
#define GW_CASE(D)                                                                                 \
    case D:                                                                                        \
        if (a.moore && a.torus) grid_walk_kernel<D, true, true><<<g, 256, 0, t->stream>>>(a, t->err);   \
        if (a.moore && !a.torus) grid_walk_kernel<D, true, false><<<g, 256, 0, t->stream>>>(a, t->err); \
        if (!a.moore && a.torus) grid_walk_kernel<D, false, true><<<g, 256, 0, t->stream>>>(a, t->err); \
        if (!a.moore && !a.torus) grid_walk_kernel<D, false, false><<<g, 256, 0, t->stream>>>(a, t->err); \
        break;
    switch (d) {
        GW_CASE(1)
        GW_CASE(2)
        GW_CASE(3)
        GW_CASE(4)
    }
#undef GW_CASE
    AMB_TRY_CUDA(cudaGetLastError());
    return AMB_OK;
}

}  // extern "C"
