// noalloc.cu -- the counting-sort cell index for callers that cannot allocate
// device memory: all of its scratch (cell counts, slot cursors, look-back
// state, error word) lives in one file-scope device array sized for grids of
// up to kStaticMaxCells cells, which every GPU that loads the library keeps
// until the process exits.
#include <mutex>

#include "amb_internal.cuh"

namespace amb {

constexpr uint32_t kStaticMaxCells = 1u << 20;  // L * L <= 1,048,576 (L <= 1024)
constexpr uint32_t kStaticTiles = (kStaticMaxCells + 4095u) / 4096u;

// byte layout of the array (each part 256-byte aligned)
constexpr size_t kOffCnt = 0;
constexpr size_t kOffCursor = kOffCnt + (size_t)kStaticMaxCells * 4u;
constexpr size_t kOffStatus = kOffCursor + (size_t)kStaticMaxCells * 4u;
constexpr size_t kOffTickets = kOffStatus + (((size_t)kStaticTiles * 8u + 255u) & ~(size_t)255u);
constexpr size_t kOffErr = kOffTickets + 256u;
constexpr size_t kStaticBytes = kOffErr + 256u;  // about 8 MiB

// Every call first clears, in stream order, the look-back words, both ticket
// counters and the error word (one contiguous stretch of 2,308 bytes), so a
// call never depends on what an earlier call, or any host-side count of
// calls, left behind: each call runs its scan with the same ticket parity and
// epoch.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticSlot {
    unsigned char *base = nullptr;  // device address of g_static_scratch on this device
};

static std::mutex g_static_mu;
static StaticSlot g_static_slots[64];

}  // namespace amb

using namespace amb;

extern "C" amb_status amb_cell_index_noalloc(const int32_t *x, const int32_t *y, uint32_t n, uint32_t L,
                                             int32_t *start, int32_t *ids, void *cuda_stream, int sync)
{
    if ((!x || !y || !ids) && n) return fail(AMB_EINVAL, "null pointer");
    if (!start) return fail(AMB_EINVAL, "null pointer");
    if (L < 1) return fail(AMB_EINVAL, "L must be >= 1");
    if ((uint64_t)L * L > kStaticMaxCells)
        return fail(AMB_EINVAL, "L*L = %llu exceeds the %u cells of the static scratch",
                    (unsigned long long)L * L, kStaticMaxCells);
    if (n > 0x7FFFFFFFu) return fail(AMB_EINVAL, "n must be < 2^31");
    if (((uintptr_t)start & 15u) != 0) return fail(AMB_EINVAL, "start must be 16-byte aligned");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return fail(AMB_ECUDA, "no usable current device");
    unsigned char *base;
    {
        // once per device, with that device current: the device address of
        // the array (host code cannot use the symbol itself)
        std::lock_guard<std::mutex> lock(g_static_mu);
        StaticSlot &slot = g_static_slots[dev];
        if (!slot.base) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess)
                return fail(AMB_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
            slot.base = static_cast<unsigned char *>(p);
        }
        base = slot.base;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int32_t *cnt = reinterpret_cast<int32_t *>(base + kOffCnt);
    int32_t *cursor = reinterpret_cast<int32_t *>(base + kOffCursor);
    uint64_t *status = reinterpret_cast<uint64_t *>(base + kOffStatus);
    unsigned long long *tickets = reinterpret_cast<unsigned long long *>(base + kOffTickets);
    uint32_t *err = reinterpret_cast<uint32_t *>(base + kOffErr);
    // look-back words ("not ready"), tickets and error word of the last call
    AMB_TRY_CUDA(cudaMemsetAsync(base + kOffStatus, 0, kOffErr + sizeof(uint32_t) - kOffStatus, s));
    AMB_TRY(launch_cell_index_raw(x, y, n, L, start, ids, cnt, cursor, status, tickets, 0u, 1u, err, s));
    if (!sync) return AMB_OK;
    uint32_t h = 0;
    AMB_TRY_CUDA(cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s));
    AMB_TRY_CUDA(cudaStreamSynchronize(s));
    if (h & ERR_TIMEOUT) return fail(AMB_ETIMEOUT, "look-back wait ran out");
    if (h & ERR_RANGE) return fail(AMB_EINVAL, "some coordinates were outside [0, L)");
    return AMB_OK;
}
