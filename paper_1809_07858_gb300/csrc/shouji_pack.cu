// shouji_pack: ASCII sequences -> bit-sliced 2-bit planes (+ optional N mask).
//
// The accelerator of the paper compares bases with XOR on an encoded form of
// both sequences (Sec. 2.3).  Here the encoding is also a transposition: one
// 32-bit output word holds one position of 32 sequences, so the filter works
// on 32 pairs per instruction.  Base codes come from bits 2 and 1 of the
// ASCII byte: A=00, C=01, G=11, T=10 (hi, lo); 'N' is flagged separately.
//
// One CTA of 256 threads packs 256 sequences = 8 lanes of a 1024-sequence
// tile.  Phase 1 stages the 256 rows in shared memory (rows padded to whole
// words, 4 words of skew per 32 rows so that phase 2 is free of bank
// conflicts).  Phase 2: a thread owns (lane, 4 consecutive positions); it
// reads one word (4 bases) of each of the lane's 32 sequences, gathers bit 2
// / bit 1 / is-'N' of every byte into byte-sliced words with shifts and
// masks, and a 4x4 byte transpose (PRMT) turns them into the four output
// words of each plane.  Stores are 32-byte (N mask) or 64-byte (planes)
// contiguous segments.
#include "shouji_internal.cuh"

namespace shouji {
namespace {

constexpr int kPackThreads = 256;
constexpr int kPackSeqs = 256;  // 8 lanes

__device__ __forceinline__ int row_word(int r, int W) { return r * W + 4 * (r >> 5); }

// 4x4 byte transpose: out[q] byte u = in[u] byte q.
__device__ __forceinline__ void transpose4x4(uint32_t y0, uint32_t y1, uint32_t y2,
                                             uint32_t y3, uint32_t out[4])
{
    uint32_t a = __byte_perm(y0, y1, 0x5140);
    uint32_t b = __byte_perm(y0, y1, 0x7362);
    uint32_t c = __byte_perm(y2, y3, 0x5140);
    uint32_t d = __byte_perm(y2, y3, 0x7362);
    out[0] = __byte_perm(a, c, 0x5410);
    out[1] = __byte_perm(a, c, 0x7632);
    out[2] = __byte_perm(b, d, 0x5410);
    out[3] = __byte_perm(b, d, 0x7632);
}

// Bit 7 of each byte of the result = that byte of w equals 'N' (0x4E).
__device__ __forceinline__ uint32_t n_bytes(uint32_t w)
{
    uint32_t x = w ^ 0x4E4E4E4Eu;
    uint32_t t = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
    return ~t & 0x80808080u;
}

template <bool WITH_N>
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const uint8_t *__restrict__ seqs, uint64_t stride, size_t n, int m,
            uint32_t *__restrict__ packed, uint32_t *__restrict__ nmask, int word_rows)
{
    extern __shared__ uint32_t sm[];
    const int W = (m + 3) >> 2;  // words per staged row
    const size_t seq0 = (size_t)blockIdx.x * kPackSeqs;
    const size_t tile = seq0 / kTile;
    const int lane0 = (int)((seq0 % kTile) / 32);

    // Phase 1: stage rows seq0 .. seq0+255 (zeros past n).
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (word_rows) {
        // Whole words inside the row are loaded as words; a partial last word
        // (m % 4 != 0) byte by byte, so nothing past byte m-1 is read.
        const int Wfull = m >> 2;
        for (int r = warp; r < kPackSeqs; r += kPackThreads / 32) {
            uint32_t *dst = sm + row_word(r, W);
            const size_t s = seq0 + r;
            const uint32_t *src = (const uint32_t *)(seqs + s * stride);
            for (int j = ln; j < W; j += 32) {
                uint32_t x = 0u;
                if (s < n) {
                    if (j < Wfull) {
                        x = __ldg(src + j);
                    } else {
                        const uint8_t *sb = (const uint8_t *)src;
                        for (int k = 0; 4 * j + k < m; ++k)
                            x |= (uint32_t)__ldg(sb + 4 * j + k) << (8 * k);
                    }
                }
                dst[j] = x;
            }
        }
    } else {
        for (int r = warp; r < kPackSeqs; r += kPackThreads / 32) {
            uint8_t *dst = (uint8_t *)(sm + row_word(r, W));
            size_t s = seq0 + r;
            const uint8_t *src = seqs + s * stride;
            for (int j = ln; j < 4 * W; j += 32)
                dst[j] = (s < n && j < m) ? __ldg(src + j) : (uint8_t)0;
        }
    }
    __syncthreads();

    // Phase 2.
    for (int item = threadIdx.x; item < 8 * W; item += kPackThreads) {
        const int l = item & 7, j = item >> 3;
        uint32_t yh[4], yl[4], yn[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            uint32_t h = 0, lo = 0, nn = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int s = 8 * t + u;
                const uint32_t w = sm[row_word(32 * l + s, W) + j];
                // bit 2 -> bit u, bit 1 -> bit u, bit 7 (is N) -> bit u of each byte
                h |= ((w >> 2) & 0x01010101u) << u;
                lo |= ((w >> 1) & 0x01010101u) << u;
                if (WITH_N)
                    nn |= (n_bytes(w) >> 7) << u;
            }
            yh[t] = h;
            yl[t] = lo;
            yn[t] = nn;
        }
        uint32_t H[4], L[4], N[4];
        transpose4x4(yh[0], yh[1], yh[2], yh[3], H);
        transpose4x4(yl[0], yl[1], yl[2], yl[3], L);
        if (WITH_N)
            transpose4x4(yn[0], yn[1], yn[2], yn[3], N);
        const int lane = lane0 + l;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int p = 4 * j + q;
            if (p < m) {
                const size_t wi = (tile * (size_t)m + p) * 32 + lane;
                reinterpret_cast<uint2 *>(packed)[wi] = make_uint2(H[q], L[q]);
                if (WITH_N)
                    nmask[wi] = N[q];
            }
        }
    }
}

}  // namespace

cudaError_t launch_pack(const uint8_t *seqs, uint64_t stride, size_t n, int m,
                        uint32_t *packed, uint32_t *nmask, cudaStream_t s)
{
    const int W = (m + 3) / 4;
    const size_t smem = (size_t)kPackSeqs * W * 4 + 8 * 4 * 4;
    const size_t blocks = tiles_of(n) * (kTile / kPackSeqs);
    const int word_rows = ((uintptr_t)seqs % 4 == 0) && (stride % 4 == 0);
    cudaError_t e;
    if (nmask) {
        e = cudaFuncSetAttribute(pack_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        pack_kernel<true><<<(unsigned)blocks, kPackThreads, smem, s>>>(seqs, stride, n, m, packed, nmask, word_rows);
    } else {
        e = cudaFuncSetAttribute(pack_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        pack_kernel<false><<<(unsigned)blocks, kPackThreads, smem, s>>>(seqs, stride, n, m, packed, nullptr, word_rows);
    }
    return cudaGetLastError();
}

}  // namespace shouji
