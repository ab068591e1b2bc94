// shouji_compact_noalloc: survivor compaction for callers that cannot call
// cudaMalloc.
//
// shouji_compact needs a small device workspace (one uint32 per slice of
// 32768 pairs) that the caller allocates.  Some callers have no way to do
// that: a host program whose device memory is owned by another allocator
// (a framework's pool with a fixed budget, an embedding application that
// hands this library only its input and output buffers), or a latency-bound
// loop that must not call cudaMalloc / cudaFree because they can synchronize
// the whole device.  For them this variant keeps its workspace in a
// file-scope __device__ array of fixed size instead.
//
// The array is a host-side stand-in in host code, not a device address, so
// the host never passes it to a kernel directly.  Its device address belongs
// to a CUDA context (the module holding the array is loaded once per
// context), not to a device: after cudaDeviceReset the device gets a new
// primary context, and a program may also make its own driver-API context
// current on the same GPU.  So the address is looked up with
// cudaGetSymbolAddress once per context, with that context current, and
// cached under the context's unique id (cuCtxGetId; ids are never reused
// within a process).  A call in a context not seen before looks the address
// up again.  The array lives on every GPU, in every context, that has used
// this entry point, until that context is destroyed.
#include <mutex>

#include "shouji_internal.cuh"

namespace shouji {
namespace {

// 64 KB: one uint32 per slice of 32 * kCompactSliceWords pairs, up to
// SHOUJI_NOALLOC_MAX_PAIRS pairs.
constexpr size_t kNoallocMaxSlices = SHOUJI_NOALLOC_MAX_PAIRS / (32 * (size_t)kCompactSliceWords);

static __device__ __align__(256) uint32_t g_compact_scratch[kNoallocMaxSlices];

// Driver entry points, taken through the runtime so that the library needs
// no link against the driver library.
using CtxGetCurrentFn = int (*)(void **ctx);
using CtxGetIdFn = int (*)(void *ctx, unsigned long long *id);

struct ScratchCache {
    std::mutex mu;
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
    bool resolved = false;
    static constexpr int kSlots = 64;
    unsigned long long ids[kSlots] = {};  // 0 = empty (context ids start at 1)
    void *addr[kSlots] = {};
    int next = 0;                         // slot replaced when all are taken
};
ScratchCache g_cache;

// Unique id of the context current on this thread (0 when none or when the
// driver entry points are missing).
unsigned long long current_context_id()
{
    if (!g_cache.resolved) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_cache.get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            g_cache.get_id = reinterpret_cast<CtxGetIdFn>(f);
        g_cache.resolved = true;
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!g_cache.get_current || !g_cache.get_id || g_cache.get_current(&ctx) != 0 || !ctx ||
        g_cache.get_id(ctx, &id) != 0)
        return 0;
    return id;
}

// Device address of g_compact_scratch in the current context: looked up
// with the context current on its first use, then taken from the cache.
cudaError_t scratch_address(void **out)
{
    std::lock_guard<std::mutex> lock(g_cache.mu);
    unsigned long long id = current_context_id();
    if (id) {
        for (int i = 0; i < ScratchCache::kSlots; ++i)
            if (g_cache.ids[i] == id) {
                *out = g_cache.addr[i];
                return cudaSuccess;
            }
    }
    void *p = nullptr;
    // Makes the runtime's context current when none was (its first call on
    // this thread), so the id read after it names the context of p.
    cudaError_t e = cudaGetSymbolAddress(&p, g_compact_scratch);
    if (e != cudaSuccess)
        return e;
    id = current_context_id();
    if (id) {
        const int slot = g_cache.next;
        g_cache.next = (slot + 1) % ScratchCache::kSlots;
        g_cache.ids[slot] = id;
        g_cache.addr[slot] = p;
    }
    *out = p;
    return cudaSuccess;
}

}  // namespace
}  // namespace shouji

using namespace shouji;

extern "C" {

shouji_status shouji_compact_noalloc(const uint32_t *accept, size_t n_pairs,
                                     uint32_t *out_idx, uint32_t *out_n, void *stream)
{
    if (n_pairs > SHOUJI_NOALLOC_MAX_PAIRS)
        return SHOUJI_EINVAL;
    if (n_pairs == 0) {
        if (out_n)
            return cuda_status(cudaMemsetAsync(out_n, 0, sizeof(uint32_t), (cudaStream_t)stream));
        return SHOUJI_OK;
    }
    if (!accept || !out_idx || !out_n)
        return SHOUJI_EINVAL;
    void *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess)
        return cuda_status(e);
    // The kernels write every slice sum before reading it: nothing in the
    // scratch needs to start at zero.
    return cuda_status(launch_compact(accept, n_pairs, out_idx, out_n, scratch,
                                      (cudaStream_t)stream));
}

}  // extern "C"
