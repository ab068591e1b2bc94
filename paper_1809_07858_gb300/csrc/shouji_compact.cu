// shouji_compact: indices of the accepted pairs, in input order.
//
// The paper's accelerator returns one result bit per pair, in input order,
// and the host picks the pairs that go on to alignment (Sec. 2.3).  Here the
// selection runs on the device in three launches over the accept bit-mask:
//   1. count:  each CTA sums the popcounts of its 1024-word slice;
//   2. scan:   one CTA turns the per-slice sums into exclusive offsets and
//              writes the total (the workspace holds one uint32 per slice);
//   3. write:  each CTA re-reads its slice and ranks every thread's four
//              words with a CTA scan; then each warp walks its 128 words in
//              order, and for each word its lanes write the indices of the
//              word's set bits with one coalesced store (lane b writes bit b
//              at the word's offset plus the bits below b).
// No CTA waits on another, so nothing can spin.
#include "shouji_internal.cuh"

namespace shouji {
namespace {

constexpr int kCThreads = 256;
constexpr int kWordsPerThread = kCompactSliceWords / kCThreads;  // 4
constexpr int kSliceWords = kCompactSliceWords;                  // 1024 words = 32768 pairs

__device__ __forceinline__ uint32_t load_word(const uint32_t *accept, size_t wi,
                                              size_t n_words, size_t n_pairs)
{
    if (wi >= n_words)
        return 0u;
    uint32_t w = __ldg(accept + wi);
    const size_t first = wi * 32;
    if (n_pairs - first < 32)
        w &= (1u << (n_pairs - first)) - 1u;
    return w;
}

// Inclusive scan of one value per thread across the CTA; returns the
// inclusive prefix and writes the CTA total.
__device__ __forceinline__ uint32_t cta_inclusive_scan(uint32_t x, uint32_t *total)
{
    __shared__ uint32_t warp_sums[kCThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < kCThreads / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o)
                s += y;
        }
        if (lane < kCThreads / 32)
            warp_sums[lane] = s;
    }
    __syncthreads();
    if (warp > 0)
        x += warp_sums[warp - 1];
    *total = warp_sums[kCThreads / 32 - 1];
    __syncthreads();
    return x;
}

__global__ void __launch_bounds__(kCThreads)
compact_count(const uint32_t *__restrict__ accept, size_t n_pairs, size_t n_words,
              uint32_t *__restrict__ slice_sums)
{
    const size_t w0 = (size_t)blockIdx.x * kSliceWords;
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < kWordsPerThread; ++i)
        c += __popc(load_word(accept, w0 + (size_t)i * kCThreads + threadIdx.x, n_words, n_pairs));
    uint32_t total;
    cta_inclusive_scan(c, &total);
    if (threadIdx.x == 0)
        slice_sums[blockIdx.x] = total;
}

// accumulate = 0: *out_n = total.  accumulate = 1: the offsets start at the
// value already in *out_n and *out_n grows by the total (chunked runs).
__global__ void __launch_bounds__(kCThreads)
compact_scan(uint32_t *__restrict__ slice_sums, uint32_t n_slices, uint32_t *__restrict__ out_n,
             int accumulate)
{
    uint32_t carry = accumulate ? *out_n : 0u;
    __syncthreads();
    for (uint32_t base = 0; base < n_slices; base += kCThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t x = i < n_slices ? slice_sums[i] : 0u;
        uint32_t total;
        const uint32_t inc = cta_inclusive_scan(x, &total);
        if (i < n_slices)
            slice_sums[i] = carry + inc - x;  // exclusive offset
        carry += total;
    }
    if (threadIdx.x == 0)
        *out_n = carry;
}

__global__ void __launch_bounds__(kCThreads)
compact_write(const uint32_t *__restrict__ accept, size_t n_pairs, size_t n_words,
              const uint32_t *__restrict__ slice_offsets, uint32_t *__restrict__ out_idx,
              uint32_t pair_base)
{
    // Thread t owns words w0 + 4t .. w0 + 4t + 3 (consecutive), so the order
    // of threads is the order of pairs.
    const int lane = threadIdx.x & 31;
    const size_t w0 = (size_t)blockIdx.x * kSliceWords + (size_t)threadIdx.x * kWordsPerThread;
    uint32_t words[kWordsPerThread], at[kWordsPerThread];
    uint32_t c = 0;
#pragma unroll
    for (int i = 0; i < kWordsPerThread; ++i) {
        words[i] = load_word(accept, w0 + i, n_words, n_pairs);
        at[i] = c;
        c += __popc(words[i]);
    }
    uint32_t total;
    const uint32_t inc = cta_inclusive_scan(c, &total);
    const uint32_t pos = slice_offsets[blockIdx.x] + inc - c;
#pragma unroll
    for (int i = 0; i < kWordsPerThread; ++i)
        at[i] += pos;
    // Word by word across the warp, in pair order: owner lane o, word i.
    const uint32_t below = (1u << lane) - 1u;
    const size_t warp_w0 = w0 - (size_t)lane * kWordsPerThread;
    for (int o = 0; o < 32; ++o) {
#pragma unroll
        for (int i = 0; i < kWordsPerThread; ++i) {
            const uint32_t w = __shfl_sync(0xFFFFFFFFu, words[i], o);
            if (!w)
                continue;
            const uint32_t base = __shfl_sync(0xFFFFFFFFu, at[i], o);
            if ((w >> lane) & 1u)
                out_idx[base + __popc(w & below)] =
                    pair_base + (uint32_t)((warp_w0 + (size_t)o * kWordsPerThread + i) * 32) +
                    (uint32_t)lane;
        }
    }
}

}  // namespace

size_t compact_workspace_bytes(size_t n_pairs)
{
    const size_t n_words = groups_of(n_pairs);
    const size_t slices = (n_words + kSliceWords - 1) / kSliceWords;
    return ((slices * sizeof(uint32_t)) + 15) / 16 * 16;
}

cudaError_t launch_compact(const uint32_t *accept, size_t n_pairs, uint32_t *out_idx,
                           uint32_t *out_n, void *workspace, cudaStream_t s)
{
    return launch_compact_append(accept, n_pairs, 0u, out_idx, out_n, 0, workspace, s);
}

cudaError_t launch_compact_append(const uint32_t *accept, size_t n_pairs, uint32_t pair_base,
                                  uint32_t *out_idx, uint32_t *total, int accumulate,
                                  void *workspace, cudaStream_t s)
{
    const size_t n_words = groups_of(n_pairs);
    const size_t slices = (n_words + kSliceWords - 1) / kSliceWords;
    uint32_t *sums = static_cast<uint32_t *>(workspace);
    compact_count<<<(unsigned)slices, kCThreads, 0, s>>>(accept, n_pairs, n_words, sums);
    compact_scan<<<1, kCThreads, 0, s>>>(sums, (uint32_t)slices, total, accumulate);
    compact_write<<<(unsigned)slices, kCThreads, 0, s>>>(accept, n_pairs, n_words, sums, out_idx,
                                                         pair_base);
    return cudaGetLastError();
}

}  // namespace shouji
