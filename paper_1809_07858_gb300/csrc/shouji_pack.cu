// shouji_pack: ASCII sequences -> bit-sliced 2-bit planes (+ optional N mask).
//
// The accelerator of the paper compares bases with XOR on an encoded form of
// both sequences (Sec. 2.3).  Here the encoding is also a transposition: one
// 32-bit output word holds one position of 32 sequences, so the filter works
// on 32 pairs per instruction.  Base codes come from bits 2 and 1 of the
// ASCII byte: A=00, C=01, G=11, T=10 (hi, lo); 'N' is flagged separately.
//
// One CTA of 256 threads packs 256 sequences = 8 lanes of a 1024-sequence
// tile (for contiguous rows on a 16-byte boundary, a persistent CTA walks
// such blocks with double buffering and bulk copies; see
// pack_stream_kernel).  Phase 1 copies the CTA's rows into shared memory as
// one dense block (row r at byte r*m).  When the rows are contiguous in
// global memory (stride == m) the block is a single contiguous range and is
// copied with 16-byte (or 4-byte) loads, four in flight per thread;
// otherwise row by row.  Phase 2: a thread owns (lane, 4 consecutive positions); it reads one
// word (4 bases) of each of the lane's 32 sequences, gathers bit 2 / bit 1 /
// is-'N' of every byte into byte-sliced words with shifts and masks, and a
// 4x4 byte transpose (PRMT) turns them into the four output words of each
// plane.  The 32 sequences are visited in an order rotated by a per-lane
// offset so that the 32 threads of a warp hit 32 different banks; the
// output word is rotated back.  Stores are 32-byte (N mask) or 64-byte
// (planes) contiguous segments.
#include "shouji_internal.cuh"
#include "shouji_pack.cuh"

namespace shouji {
namespace {

using namespace packdev;

constexpr int kPackThreads = 256;
constexpr int kPackSeqs = 256;  // 8 lanes

enum CopyMode { kCopyVec16 = 0, kCopyVec4 = 1, kCopyRows = 2 };

// Set when a pack without an N mask read an 'N' (see shouji_unmasked_n),
// unless the caller gave a flag word of its own.
__device__ unsigned int g_pack_unmasked_n;

__device__ __forceinline__ void flag_unmasked_n(unsigned int *nflag)
{
    if (nflag)
        *nflag = 1u;
    else
        g_pack_unmasked_n = 1u;
}

// ALIGNED: m % 4 == 0, so every 4-position word of a row is word-aligned.
template <bool WITH_N, bool ALIGNED>
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const uint8_t *__restrict__ seqs, uint64_t stride, size_t n, int m,
            uint32_t *__restrict__ packed, uint32_t *__restrict__ nmask, int copy_mode,
            int rot_step, unsigned int *nflag)
{
    extern __shared__ __align__(16) uint32_t sm[];
    uint8_t *sb = reinterpret_cast<uint8_t *>(sm);
    const size_t seq0 = (size_t)blockIdx.x * kPackSeqs;
    const size_t tile = seq0 / kTile;
    const int lane0 = (int)((seq0 % kTile) / 32);
    // Blocks of the last tile may start at or past n: they stage no rows.
    const size_t left = seq0 < n ? n - seq0 : 0;
    const int rows = (int)(left < (size_t)kPackSeqs ? left : (size_t)kPackSeqs);
    const int nbytes = rows * m;                 // staged bytes holding real rows
    const int total = kPackSeqs * m + 16;        // staged bytes incl. zero padding
    const int tid = threadIdx.x;

    // Phase 1: stage rows seq0 .. seq0+rows-1 densely; zeros after them.
    if (copy_mode == kCopyVec16) {
        const uint4 *src = reinterpret_cast<const uint4 *>(seqs + seq0 * (size_t)m);
        uint4 *dst = reinterpret_cast<uint4 *>(sm);
        const int nvec = nbytes >> 4;
        int k = tid;
        for (; k + 3 * kPackThreads < nvec; k += 4 * kPackThreads) {
            const uint4 a = __ldg(src + k), b = __ldg(src + k + kPackThreads);
            const uint4 c = __ldg(src + k + 2 * kPackThreads), d = __ldg(src + k + 3 * kPackThreads);
            dst[k] = a;
            dst[k + kPackThreads] = b;
            dst[k + 2 * kPackThreads] = c;
            dst[k + 3 * kPackThreads] = d;
        }
        for (; k < nvec; k += kPackThreads)
            dst[k] = __ldg(src + k);
        for (int b = (nvec << 4) + tid; b < nbytes; b += kPackThreads)
            sb[b] = __ldg(seqs + seq0 * (size_t)m + b);
    } else if (copy_mode == kCopyVec4) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(seqs + seq0 * (size_t)m);
        const int nw = nbytes >> 2;
        int k = tid;
        for (; k + 3 * kPackThreads < nw; k += 4 * kPackThreads) {
            const uint32_t a = __ldg(src + k), b = __ldg(src + k + kPackThreads);
            const uint32_t c = __ldg(src + k + 2 * kPackThreads), d = __ldg(src + k + 3 * kPackThreads);
            sm[k] = a;
            sm[k + kPackThreads] = b;
            sm[k + 2 * kPackThreads] = c;
            sm[k + 3 * kPackThreads] = d;
        }
        for (; k < nw; k += kPackThreads)
            sm[k] = __ldg(src + k);
        for (int b = (nw << 2) + tid; b < nbytes; b += kPackThreads)
            sb[b] = __ldg(seqs + seq0 * (size_t)m + b);
    } else {
        const int warp = tid >> 5, ln = tid & 31;
        for (int r = warp; r < rows; r += kPackThreads / 32) {
            const uint8_t *src = seqs + (seq0 + r) * stride;
            for (int j = ln; j < m; j += 32)
                sb[r * m + j] = __ldg(src + j);
        }
    }
    for (int b = nbytes + tid; b < total; b += kPackThreads)
        sb[b] = 0;
    __syncthreads();

    const uint32_t seen =
        pack_transpose<WITH_N, ALIGNED>(sm, m, m, tile, lane0, packed, nmask, rot_step, kPackThreads);
    if (!WITH_N && __syncthreads_or(has_n_bytes(seen)) && tid == 0)
        flag_unmasked_n(nflag);
}

// Bounded waits of pack_stream_kernel that ran out (see shouji_wait_failures).
__device__ unsigned int g_pack_wait_failures;

// Contiguous rows on a 16-byte boundary (the common case): a persistent,
// double-buffered form.  Each CTA walks blocks blockIdx.x, +gridDim.x, ...;
// while it transposes block i from one buffer, one bulk copy (the TMA unit)
// brings the rows of block i+1 into the other, completing on that buffer's
// mbarrier, so the loads of the next block overlap the transposition of this
// one.  The copy moves the block's bytes rounded down to 16; the threads add
// the last few bytes of a partial block and the zero padding after the rows.
// A wait that runs out (a copy that never lands) ends the CTA and counts one
// failure; the CTA first waits, bounded too, for its other copy in flight.
// extra_tx is 0 except in the self-test of that path, which announces each
// copy 16 bytes longer than it is so that no wait can complete.
template <bool WITH_N, bool ALIGNED>
__global__ void __launch_bounds__(kPackThreads)
pack_stream_kernel(const uint8_t *__restrict__ seqs, size_t n, int m,
                   uint32_t *__restrict__ packed, uint32_t *__restrict__ nmask, int rot_step,
                   size_t n_blocks, int buf_bytes, uint32_t extra_tx, unsigned int *nflag)
{
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ __align__(8) uint64_t full[2];
    uint8_t *bufs = reinterpret_cast<uint8_t *>(sm);
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    // staged bytes holding real rows; blocks of the last tile may start at or
    // past n and stage none
    auto row_bytes = [&](size_t blk) -> int {
        const size_t seq0 = blk * kPackSeqs;
        const size_t left = seq0 < n ? n - seq0 : 0;
        return (int)(left < (size_t)kPackSeqs ? left : (size_t)kPackSeqs) * m;
    };
    auto issue = [&](size_t blk, int b) {  // one thread
        const uint32_t bytes = (uint32_t)row_bytes(blk) & ~15u;
        mbar_arrive_expect_tx(&full[b], bytes + extra_tx);
        if (bytes)
            bulk_copy_g2s(bufs + (size_t)b * buf_bytes, seqs + blk * kPackSeqs * (size_t)m, bytes,
                          &full[b]);
    };

    size_t blk = blockIdx.x;
    if (tid == 0 && blk < n_blocks)
        issue(blk, 0);
    uint32_t parity = 0;  // bit b: parity of the phase of full[b] to wait for
    for (int i = 0; blk < n_blocks; ++i, blk += gridDim.x) {
        const int b = i & 1;
        const size_t next = blk + gridDim.x;
        if (tid == 0 && next < n_blocks) {
            fence_proxy_async_smem();  // buffer b^1 was read in the last round
            issue(next, b ^ 1);
        }
        const bool ok = mbar_wait_bounded(&full[b], (parity >> b) & 1u);
        parity ^= 1u << b;
        uint8_t *buf = bufs + (size_t)b * buf_bytes;
        const int nbytes = row_bytes(blk);
        const size_t seq0 = blk * kPackSeqs;
        for (int x = (nbytes & ~15) + tid; x < buf_bytes; x += kPackThreads)
            buf[x] = x < nbytes ? __ldg(seqs + seq0 * (size_t)m + x) : (uint8_t)0;
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicAdd(&g_pack_wait_failures, 1u);
                if (next < n_blocks)
                    mbar_wait_bounded(&full[b ^ 1], (parity >> (b ^ 1)) & 1u);
            }
            return;
        }
        const uint32_t seen = pack_transpose<WITH_N, ALIGNED>(
            reinterpret_cast<const uint32_t *>(buf), m, m, seq0 / kTile,
            (int)((seq0 % kTile) / 32), packed, nmask, rot_step, kPackThreads);
        // the buffer may be refilled after this barrier
        if (WITH_N)
            __syncthreads();
        else if (__syncthreads_or(has_n_bytes(seen)) && tid == 0)
            flag_unmasked_n(nflag);
    }
}

template <bool WITH_N, bool ALIGNED>
cudaError_t launch_stream_ta(const uint8_t *seqs, size_t n, int m, uint32_t *packed,
                             uint32_t *nmask, int rot, cudaStream_t s, uint32_t extra_tx = 0,
                             unsigned int *nflag = nullptr)
{
    // one buffer: 256 rows of m bytes and 16 bytes of zero padding, rounded
    // up to 128 bytes
    const int buf_bytes = (kPackSeqs * m + 16 + 127) / 128 * 128;
    const size_t smem = 2 * (size_t)buf_bytes;
    const size_t n_blocks = tiles_of(n) * (kTile / kPackSeqs);
    cudaError_t e = cudaFuncSetAttribute(pack_stream_kernel<WITH_N, ALIGNED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
             &per_sm, pack_stream_kernel<WITH_N, ALIGNED>, kPackThreads, smem)) != cudaSuccess)
        return e;
    const size_t full = (size_t)sms * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(n_blocks < full ? n_blocks : full);
    pack_stream_kernel<WITH_N, ALIGNED><<<grid, kPackThreads, smem, s>>>(
        seqs, n, m, packed, nmask, rot, n_blocks, buf_bytes, extra_tx, nflag);
    return cudaGetLastError();
}

template <bool WITH_N>
cudaError_t launch_stream_t(const uint8_t *seqs, size_t n, int m, uint32_t *packed,
                            uint32_t *nmask, int rot, cudaStream_t s, unsigned int *nflag)
{
    if (m % 4 == 0)
        return launch_stream_ta<WITH_N, true>(seqs, n, m, packed, nmask, rot, s, 0, nflag);
    return launch_stream_ta<WITH_N, false>(seqs, n, m, packed, nmask, rot, s, 0, nflag);
}

template <bool WITH_N>
cudaError_t launch_pack_t(const uint8_t *seqs, uint64_t stride, size_t n, int m,
                          uint32_t *packed, uint32_t *nmask, cudaStream_t s, unsigned int *nflag)
{
    const size_t smem = (size_t)kPackSeqs * m + 16;
    const size_t blocks = tiles_of(n) * (kTile / kPackSeqs);
    int mode = kCopyRows;
    if (stride == (uint64_t)m) {
        if ((uintptr_t)seqs % 16 == 0)
            mode = kCopyVec16;
        else if ((uintptr_t)seqs % 4 == 0 && m % 4 == 0)
            mode = kCopyVec4;
    }
    const int rot = rotation_step(m);
    cudaError_t e;
    if (mode == kCopyVec16)
        return launch_stream_t<WITH_N>(seqs, n, m, packed, nmask, rot, s, nflag);
    if (m % 4 == 0) {
        e = cudaFuncSetAttribute(pack_kernel<WITH_N, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        pack_kernel<WITH_N, true><<<(unsigned)blocks, kPackThreads, smem, s>>>(
            seqs, stride, n, m, packed, nmask, mode, rot, nflag);
    } else {
        e = cudaFuncSetAttribute(pack_kernel<WITH_N, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        pack_kernel<WITH_N, false><<<(unsigned)blocks, kPackThreads, smem, s>>>(
            seqs, stride, n, m, packed, nmask, mode, rot, nflag);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack(const uint8_t *seqs, uint64_t stride, size_t n, int m,
                        uint32_t *packed, uint32_t *nmask, cudaStream_t s, unsigned int *nflag)
{
    if (nmask)
        return launch_pack_t<true>(seqs, stride, n, m, packed, nmask, s, nullptr);
    return launch_pack_t<false>(seqs, stride, n, m, packed, nmask, s, nflag);
}

cudaError_t take_pack_unmasked_n(uint32_t *seen)
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_pack_unmasked_n, sizeof v);
    if (e == cudaSuccess && v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_pack_unmasked_n, &zero, sizeof zero);
    }
    *seen = v;
    return e;
}

cudaError_t take_wait_failures(uint32_t *count)
{
    cudaError_t e = cudaDeviceSynchronize();
    unsigned int v = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyFromSymbol(&v, g_pack_wait_failures, sizeof v);
    if (e == cudaSuccess && v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_pack_wait_failures, &zero, sizeof zero);
    }
    uint32_t fused = 0;
    if (e == cudaSuccess)
        e = take_fused_wait_failures(&fused);
    *count = v + fused;
    return e;
}

cudaError_t selftest_pack_wait(uint32_t *failures)
{
    // 1024 sequences of 4 bases: one tile, 4 blocks, one per CTA
    constexpr size_t n = 1024;
    constexpr int m = 4;
    *failures = 0;
    uint32_t before = 0;
    cudaError_t e = take_wait_failures(&before);
    if (e != cudaSuccess)
        return e;
    uint8_t *seqs = nullptr;
    uint32_t *packed = nullptr;
    if ((e = cudaMalloc(&seqs, n * m)) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(&packed, tiles_of(n) * m * 64 * sizeof(uint32_t))) == cudaSuccess &&
        (e = cudaMemset(seqs, 'A', n * m)) == cudaSuccess &&
        (e = launch_stream_ta<false, true>(seqs, n, m, packed, nullptr, rotation_step(m), 0,
                                           16u)) == cudaSuccess)
        e = take_wait_failures(failures);
    cudaFree(packed);
    cudaFree(seqs);
    return e;
}

}  // namespace shouji
