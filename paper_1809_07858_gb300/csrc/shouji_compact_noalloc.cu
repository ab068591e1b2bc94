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
// the host never passes it to a kernel directly: once per device, with that
// device current, the first call asks cudaGetSymbolAddress for the device
// address and caches it.  The array lives on every GPU that loads the
// library until the process exits.
#include <atomic>

#include "shouji_internal.cuh"

namespace shouji {
namespace {

constexpr int kNoallocMaxDevices = 64;
// 64 KB: one uint32 per slice of 32 * kCompactSliceWords pairs, up to
// SHOUJI_NOALLOC_MAX_PAIRS pairs.
constexpr size_t kNoallocMaxSlices = SHOUJI_NOALLOC_MAX_PAIRS / (32 * (size_t)kCompactSliceWords);

static __device__ __align__(256) uint32_t g_compact_scratch[kNoallocMaxSlices];

std::atomic<void *> g_scratch_addr[kNoallocMaxDevices];

// Device address of g_compact_scratch on the current device (set-up on the
// first call per device).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return cudaErrorInvalidDevice;
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_compact_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[dev].store(p, std::memory_order_release);
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
