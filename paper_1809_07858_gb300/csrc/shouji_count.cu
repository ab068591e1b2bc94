// shouji_count: local and semi-global ("glocal") counting of the Shouji
// bit-vectors (Sec. 2.2.3 and Supplementary Sec. 8, Fig. 6(c) of the paper).
//
// The filter counts every one of the Shouji bit-vector (global mode).  For
// local alignment the runs of ones at the two ends of the vector are not
// edits of the aligned part and are left out; for glocal (semi-global)
// alignment, the run at one end.  This pass reads the bit-sliced vectors
// that shouji_filter writes (out_vectors) and recounts them: one thread per
// group of 32 pairs walks the m position words of its group (coalesced
// across the warp) and keeps four bit-sliced counters per group: all ones,
// ones before the first zero, ones since the last zero, and whether a zero
// was seen.  A vector without a zero counts m in every mode.
#include "shouji_internal.cuh"

namespace shouji {
namespace {

constexpr int kCountThreads = 128;

// 8-bit bit-sliced counter += x (one bit per pair).
__device__ __forceinline__ void inc(uint32_t (&c)[8], uint32_t x)
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t carry = c[k] & x;
        c[k] ^= x;
        x = carry;
    }
}

// a - b on 8-bit bit-sliced numbers (b <= a wherever the result is used).
__device__ __forceinline__ void sub(const uint32_t (&a)[8], const uint32_t (&b)[8], uint32_t (&r)[8])
{
    uint32_t borrow = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        r[k] = a[k] ^ b[k] ^ borrow;
        borrow = (~a[k] & (b[k] | borrow)) | (b[k] & borrow);
    }
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&c)[8], int b)
{
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
        v |= ((c[k] >> b) & 1u) << k;
    return v;
}

__global__ void __launch_bounds__(kCountThreads)
count_kernel(const uint32_t *__restrict__ vectors, int m, size_t n_pairs, int E,
             const uint8_t *__restrict__ E_per_pair, int mode, uint32_t *__restrict__ accept,
             uint8_t *__restrict__ count)
{
    const size_t g = (size_t)blockIdx.x * kCountThreads + threadIdx.x;
    if (g >= groups_of(n_pairs))
        return;
    const uint32_t *v = vectors + (g / kLanes) * (size_t)m * kLanes + (g % kLanes);
    uint32_t all[8], lead[8], pend[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
        all[k] = lead[k] = pend[k] = 0u;
    uint32_t seen = 0u;
    for (int c = 0; c < m; ++c) {
        const uint32_t o = __ldg(v + (size_t)c * kLanes);
        inc(all, o);
        inc(lead, o & ~seen);
        seen |= ~o;
        inc(pend, o);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            pend[k] &= o;  // a zero restarts the trailing run
    }
    uint32_t res[8], tmp[8];
    if (mode == SHOUJI_COUNT_LOCAL) {
        sub(all, lead, tmp);
        sub(tmp, pend, res);
    } else if (mode == SHOUJI_COUNT_GLOCAL_START) {
        sub(all, lead, res);
    } else if (mode == SHOUJI_COUNT_GLOCAL_END) {
        sub(all, pend, res);
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            res[k] = all[k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)  // no zero at all: the vector counts m
        res[k] = (res[k] & seen) | (all[k] & ~seen);
    const size_t first = g * 32;
    const size_t left = n_pairs - first;
    uint32_t acc = 0;
    for (int b = 0; b < 32 && (size_t)b < left; ++b) {
        const uint32_t cnt = byte_of(res, b);
        const uint32_t e = E_per_pair ? min((uint32_t)E_per_pair[first + b], (uint32_t)E) : (uint32_t)E;
        acc |= (uint32_t)(cnt <= e) << b;
        if (count)
            count[first + b] = (uint8_t)cnt;
    }
    accept[g] = acc;
}

}  // namespace
}  // namespace shouji

using namespace shouji;

extern "C" shouji_status shouji_count(const uint32_t *vectors, uint32_t m, size_t n_pairs, int E,
                                      const uint8_t *E_per_pair, int mode, uint32_t *out_accept,
                                      uint8_t *out_count, void *stream)
{
    if (m < 1 || m > SHOUJI_MAX_M || E < 0 || E > SHOUJI_MAX_E || mode < SHOUJI_COUNT_GLOBAL ||
        mode > SHOUJI_COUNT_GLOCAL_END)
        return SHOUJI_EINVAL;
    if (n_pairs == 0)
        return SHOUJI_OK;
    if (!vectors || !out_accept)
        return SHOUJI_EINVAL;
    const size_t groups = groups_of(n_pairs);
    count_kernel<<<(unsigned)((groups + kCountThreads - 1) / kCountThreads), kCountThreads, 0,
                   (cudaStream_t)stream>>>(vectors, (int)m, n_pairs, E, E_per_pair, mode,
                                           out_accept, out_count);
    return cuda_status(cudaGetLastError());
}
