// Internal declarations shared by the translation units of libshouji.so.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "shouji.h"

namespace shouji {

constexpr int kLanes = 32;            // 32-bit words per tile position
constexpr int kTile = 32 * kLanes;    // sequences per tile (SHOUJI_TILE)

__host__ __device__ inline size_t tiles_of(size_t n) { return (n + kTile - 1) / kTile; }
__host__ __device__ inline size_t groups_of(size_t n) { return (n + 31) / 32; }

// Remember a failed CUDA call for shouji_last_cuda_error() and map it to a
// status code.
shouji_status cuda_status(cudaError_t e);

// Launchers (argument checks are done by the C-ABI layer).  Without an N
// mask the pack sets *nflag (device), or the library's flag when nflag is
// null, when it reads an 'N'.
cudaError_t launch_pack(const uint8_t *seqs, uint64_t stride, size_t n, int m,
                        uint32_t *packed, uint32_t *nmask, cudaStream_t s,
                        unsigned int *nflag = nullptr);
// Synchronizes the device, then reads and resets the count of bounded
// device waits that ran out (pack staging and the fused pack + filter).
cudaError_t take_wait_failures(uint32_t *count);

// Largest threshold of the fused pack + filter kernel (its filter warps
// have 128 registers).
#define SHOUJI_FUSED_MAX_E 5
// Whether the fused kernel takes length m and threshold E (the two staging
// rings must hold at least two 256-row blocks each).
bool pack_filter_fusable(int m, int E);
// Pack of both sets and the filter in one kernel; rows contiguous (stride
// m) on 16-byte boundaries, no N masks or per-pair thresholds (checked by
// the caller).  cudaErrorNotSupported, with nothing launched, when the
// kernel does not apply (pack_filter_fusable, or a compiled register count
// other than the one its register split assumes).  ring_mode: packed_r and
// packed_t are per-CTA rings of pack_filter_ring_words() words each instead
// of packed outputs.
cudaError_t launch_pack_filter(const uint8_t *reads, const uint8_t *refs, size_t n, int m, int E,
                               uint32_t *packed_r, uint32_t *packed_t, uint32_t *accept,
                               uint8_t *count, cudaStream_t s, bool ring_mode = false);
// CTAs of the fused kernel for n pairs on a GPU of `sms` SMs, and the words of
// one side's rings in ring mode (a queue slot's tile per CTA and slot).
size_t pack_filter_grid(size_t n, int sms);
size_t pack_filter_ring_words(size_t n, int m, int sms);
// Whether launch_pack_filter would run the fused kernel for length m and
// threshold E (pack_filter_fusable and the compiled register count).
cudaError_t pack_filter_kernel_applies(int m, int E, bool *applies);
// Read and reset the flags that packs without N masks set when they read an
// 'N' (no sync): standalone packs, the fused kernel, the batched packs.
cudaError_t take_pack_unmasked_n(uint32_t *seen);
cudaError_t take_fused_unmasked_n(uint32_t *seen);
cudaError_t take_batch_unmasked_n(uint32_t *seen);
// Synchronizes the device, then reads and resets all three (nonzero: seen).
cudaError_t take_unmasked_n(uint32_t *seen);
// Reads and resets the fused kernel's count of waits that ran out (no sync).
cudaError_t take_fused_wait_failures(uint32_t *count);
// Runs the pack on 1024 sequences with every staging wait made to run out;
// writes the failures counted.
cudaError_t selftest_pack_wait(uint32_t *failures);

// Measured lane-ops per SM clock of one instruction kind (SHOUJI_PROBE_*).
cudaError_t alu_probe(int op, double *rate);

struct FilterArgs {
    const uint2 *reads, *refs;               // packed pairs (hi, lo) words
    const uint32_t *reads_n, *refs_n;        // N masks or null
    const uint8_t *E_per_pair;               // per-pair thresholds or null
    uint32_t *accept;                        // ceil(n/32) words
    uint8_t *count;                          // n bytes or null
    uint32_t *vectors;                       // bit-sliced Shouji vectors or null
    size_t n_pairs;
    int m;
};
cudaError_t launch_filter(const FilterArgs &a, int E, cudaStream_t s);

// One launcher per threshold, defined in the per-range instantiation units.
template <int E>
cudaError_t launch_filter_E(const FilterArgs &a, cudaStream_t s);

// Compaction works on slices of kCompactSliceWords accept words (32 pairs
// each); its workspace holds one uint32 per slice.
constexpr int kCompactSliceWords = 1024;
size_t compact_workspace_bytes(size_t n_pairs);
cudaError_t launch_compact(const uint32_t *accept, size_t n_pairs,
                           uint32_t *out_idx, uint32_t *out_n, void *workspace,
                           cudaStream_t s);
// Chunked form: indices are offset by pair_base; with accumulate the output
// position starts at *total and *total grows by the chunk's count.
cudaError_t launch_compact_append(const uint32_t *accept, size_t n_pairs,
                                  uint32_t pair_base, uint32_t *out_idx,
                                  uint32_t *total, int accumulate,
                                  void *workspace, cudaStream_t s);

}  // namespace shouji
