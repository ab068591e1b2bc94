// Batched filter for pairs of mixed lengths and thresholds, as one CUDA graph.
//
// The Shouji filter runs in time m (2E + 2) per pair (Eq. 2 of the paper);
// a batch mixing lengths 100/150/250 and thresholds 2..12 would, unsorted,
// make almost every bit-sliced group of 32 pairs pay for its longest and
// most tolerant member.  The batch object therefore runs, per batch:
//   classify  key = (m, E) per pair, its rank inside the bucket (CTA-local
//             histogram with warp-aggregated shared atomics, then one global
//             atomic per CTA and bucket)
//   scan      one CTA lays the buckets out: by m (each m-class on 1024-pair
//             tiles: a packed tile has one length), inside by E (each bucket
//             on 32-pair groups: a group runs one threshold), and lists the
//             buckets of every threshold with their group offsets
//   fill + scatter   slot -> pair permutation (padding slots: no pair)
//   pack      reads and refs gathered through the permutation and packed
//             into the bit-sliced layout of their m-class
//   filter    one persistent kernel per threshold E in [e_min, e_max],
//             specialised for E, walking the groups of all of its buckets
//   finalize  counts gathered back to input order, accept bits by ballot
// All launches are captured once into a CUDA graph; a run copies its
// argument block into pinned memory and launches the graph.  The launch
// shape of each threshold's kernel (CTA size, CTAs per SM, schedule) comes
// from the autotuner (shouji_batch_tune) or defaults.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "shouji_batch.cuh"
#include "shouji_pack.cuh"

namespace shouji {
namespace batch {
namespace {

// Set when a batch without N masks read an 'N' (see shouji_unmasked_n).
__device__ unsigned int g_batch_unmasked_n;

constexpr int kClsThreads = 256;
constexpr int kClsItems = 16;                       // pairs per thread
constexpr int kClsPairs = kClsThreads * kClsItems;  // pairs per chunk
constexpr int kClsCtasPerSm = 4;                    // 40 KB of shared memory each
constexpr int kPackThreads = 128;
constexpr int kPackSeqs = 128;   // 4 lanes of a tile per CTA
constexpr int kPackLanes = kPackSeqs / 32;

// Shared-memory row stride of the batch pack: m rounded up to 16 bytes, and
// moved off multiples of 32 bytes.
__host__ __device__ inline int row_stride(int m)
{
    int rs = (m + 15) & ~15;
    if (rs % 32 == 0)
        rs += 16;
    return rs;
}

// Whole 16-byte chunks of every row may be read: rows start on 16-byte
// boundaries and the stride covers the longest row rounded up to 16 bytes.
__device__ __forceinline__ bool rows_on_16_bytes(const uint8_t *seqs, uint64_t stride, int max_m)
{
    return (stride % 16 == 0) && ((uintptr_t)seqs % 16 == 0) &&
           stride >= (uint64_t)((max_m + 15) & ~15);
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------- classify
// Persistent: each CTA walks chunks of kClsPairs pairs (blockIdx.x, +gridDim.x,
// ...).  Per chunk, every pair gets its rank among the chunk's pairs of its
// bucket from a shared histogram (warp-aggregated increments); the first
// increment of a bucket lists it, and only the listed buckets are reserved
// in the global histogram (one atomic per bucket and chunk) and cleared for
// the next chunk.
__global__ void __launch_bounds__(kClsThreads)
classify_kernel(const Args *__restrict__ a, int max_m, int e_lo, int e_hi,
                uint32_t *__restrict__ hist, Tables *__restrict__ T,
                uint16_t *__restrict__ keys, uint32_t *__restrict__ ranks)
{
    __shared__ uint32_t sh[kBins];
    __shared__ uint16_t touched[kClsPairs];   // buckets a chunk's pairs fell in
    __shared__ uint32_t n_touched;
    const uint64_t n = a->n;
    const uint64_t chunks = (n + kClsPairs - 1) / kClsPairs;
    if (blockIdx.x >= chunks)
        return;
    for (int k = threadIdx.x; k < kBins; k += kClsThreads)
        sh[k] = 0u;
    if (threadIdx.x == 0)
        n_touched = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t bad = 0;
    for (uint64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        const uint64_t i0 = c * kClsPairs;
        uint16_t key[kClsItems];
        uint32_t local[kClsItems];
#pragma unroll
        for (int t = 0; t < kClsItems; ++t) {
            const uint64_t i = i0 + (uint64_t)t * kClsThreads + threadIdx.x;
            int k = -1;
            if (i < n) {
                const int m = a->lens[i];
                const int e = a->E_per_pair[i];
                if (m >= 1 && m <= max_m && e >= e_lo && e <= e_hi)
                    k = m * kMaxE + e;
                else
                    ++bad;
            }
            // warp-aggregated increment of the shared bucket counter
            const uint32_t peers = __match_any_sync(0xffffffffu, k);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if (lane == leader && k >= 0) {
                base = atomicAdd(&sh[k], (uint32_t)__popc(peers));
                if (base == 0)
                    touched[atomicAdd(&n_touched, 1u)] = (uint16_t)k;
            }
            base = __shfl_sync(0xffffffffu, base, leader);
            key[t] = k >= 0 ? (uint16_t)k : kBadKey;
            local[t] = base + __popc(peers & lanemask_lt());
        }
        __syncthreads();
        const uint32_t nt = n_touched;
        // one global reservation per bucket of this chunk
        for (uint32_t q = threadIdx.x; q < nt; q += kClsThreads) {
            const int k = touched[q];
            sh[k] = atomicAdd(&hist[k], sh[k]);
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kClsItems; ++t) {
            const uint64_t i = i0 + (uint64_t)t * kClsThreads + threadIdx.x;
            if (i < n) {
                keys[i] = key[t];
                ranks[i] = key[t] != kBadKey ? sh[key[t]] + local[t] : 0u;
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < nt; q += kClsThreads)
            sh[touched[q]] = 0u;
        if (threadIdx.x == 0)
            n_touched = 0u;
        __syncthreads();
    }
    if (bad)
        atomicAdd(&T->n_invalid, bad);
}

// ---------------------------------------------------------------- scan
__global__ void __launch_bounds__(256)
scan_kernel(const uint32_t *__restrict__ hist, Tables *__restrict__ T)
{
    __shared__ uint32_t pad_m[kMaxM];   // slots of m-class m (bucket pads to 32, tile pad)
    __shared__ uint32_t mc_of[kMaxM];
    __shared__ uint32_t start_m[kMaxM];
    __shared__ uint32_t h[kBins];       // the histogram: every pass below reads it here
    const int t = threadIdx.x;
    for (int k = t; k < kBins; k += 256)
        h[k] = hist[k];
    __syncthreads();
    static_assert(kMaxE == 32, "a lane per threshold");
    // slots of each m-class: a warp per m, a lane per E (conflict-free reads)
    const int warp = t >> 5, lane = t & 31;
    for (int m = warp; m < kMaxM; m += 8) {
        uint32_t p = m >= 1 ? (h[m * kMaxE + lane] + 31u) & ~31u : 0u;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1)
            p += __shfl_xor_sync(0xffffffffu, p, o);
        if (lane == 0)
            pad_m[m] = (p + kTile - 1) / kTile * kTile;
    }
    __syncthreads();
    if (t == 0) {
        uint32_t slot = 0, blocks = 0, nmc = 0;
        uint64_t poff = 0;
        T->mc_block[0] = 0;
        for (int m = 1; m < kMaxM; ++m) {
            start_m[m] = slot;
            mc_of[m] = nmc;
            if (pad_m[m]) {
                T->mc_m[nmc] = m;
                T->mc_slot[nmc] = slot;
                T->mc_poff[nmc] = poff;
                blocks += pad_m[m] / kPackSeqs;
                T->mc_block[nmc + 1] = blocks;
                poff += (uint64_t)(pad_m[m] / kTile) * m * kLanes;
                slot += pad_m[m];
                ++nmc;
            }
        }
        T->n_mc = nmc;
        T->total_slots = slot;
    }
    __syncthreads();
    // first slot of each bucket (m, E): the m-class start plus the padded sizes
    // of the buckets of smaller E, by an exclusive scan over the warp's lanes
    for (int m = 1 + warp; m < kMaxM; m += 8) {
        const uint32_t v = (h[m * kMaxE + lane] + 31u) & ~31u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        T->bin_slot[m * kMaxE + lane] = start_m[m] + x - v;
    }
    __syncthreads();
    if (t < kMaxE) {
        const int e = t;
        uint32_t cnt = 0, gs = 0;
        for (int m = 1; m < kMaxM; ++m) {
            const uint32_t c = h[m * kMaxE + e];
            if (c) {
                const int b = e * kMaxM + cnt;
                T->bk_m[b] = m;
                T->bk_slot[b] = T->bin_slot[m * kMaxE + e];
                T->bk_count[b] = c;
                T->bk_gstart[b] = gs;
                T->bk_mc[b] = mc_of[m];
                gs += (c + 31u) / 32u;
                ++cnt;
            }
        }
        T->ec_first[e] = e * kMaxM;
        T->ec_count[e] = cnt;
        T->ec_groups[e] = gs;
    }
}

// ---------------------------------------------------------------- permutation
__global__ void fill_kernel(const Tables *__restrict__ T, uint32_t *__restrict__ perm)
{
    const uint32_t total = T->total_slots;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < total; s += gridDim.x * blockDim.x)
        perm[s] = kNoPair;
}

__global__ void scatter_kernel(const Args *__restrict__ a, const Tables *__restrict__ T,
                               const uint16_t *__restrict__ keys,
                               const uint32_t *__restrict__ ranks, uint32_t *__restrict__ perm)
{
    const uint64_t n = a->n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint16_t k = keys[i];
        if (k != kBadKey)
            perm[T->bin_slot[k] + ranks[i]] = (uint32_t)i;
    }
}

// ---------------------------------------------------------------- pack
// blockIdx.y = 0: reads, 1: refs.  A block packs 128 slots (4 lanes of a
// tile) of one m-class; the CTAs walk the blocks blockIdx.x, +gridDim.x, ...
// This byte-gather form serves rows that are not on 16-byte boundaries and
// exits at once otherwise (pack_async_kernel packs those).
template <bool WITH_N>
__global__ void __launch_bounds__(kPackThreads)
pack_kernel(const Args *__restrict__ a, const Tables *__restrict__ T, int max_m,
            const uint32_t *__restrict__ perm, uint2 *__restrict__ preads,
            uint2 *__restrict__ prefs, uint32_t *__restrict__ nreads,
            uint32_t *__restrict__ nrefs)
{
    extern __shared__ __align__(16) uint32_t sm[];
    uint8_t *sb = reinterpret_cast<uint8_t *>(sm);
    const uint8_t *seqs = blockIdx.y ? a->refs : a->reads;
    const uint64_t stride = a->stride;
    const uint64_t *off = blockIdx.y ? a->ref_off : nullptr;  // rows at offsets
    // rows on 16-byte boundaries are packed by pack_async_kernel instead
    if (!off && rows_on_16_bytes(seqs, stride, max_m))
        return;
    const uint32_t nmc = T->n_mc;
    if (nmc == 0)
        return;
    const uint32_t total = T->mc_block[nmc];
    // the CTAs walk the blocks blockIdx.x, +gridDim.x, ...
    for (uint32_t blk = blockIdx.x; blk < total; blk += gridDim.x) {
        uint32_t lo = 0, hi = nmc;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (T->mc_block[mid] <= blk)
                lo = mid;
            else
                hi = mid;
        }
        const int m = (int)T->mc_m[lo];
        const uint32_t rel = (blk - T->mc_block[lo]) * kPackSeqs;  // slot offset in the m-class
        const uint32_t slot0 = T->mc_slot[lo] + rel;

        // Phase 1: gather the 128 rows (zeros for padding slots) into sm, row r
        // at byte r * rs, as bytes, 8 rows per warp at a time.
        const int rs = row_stride(m);
        {
            const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31;
            for (int rb = 0; rb < 32; rb += 8) {
                const int r0 = warp * 32 + rb;
                uint32_t pair[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    pair[k] = perm[slot0 + r0 + k];
                uint8_t v[8][8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const bool ok = pair[k] != kNoPair;
                    const uint64_t p = ok ? pair[k] : 0;
                    const uint8_t *src = seqs + (off ? (ok ? off[p] : 0) : p * stride);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = ln + 32 * q;
                        v[k][q] = (ok && j < m) ? __ldg(src + j) : (uint8_t)0;
                    }
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    uint8_t *dst = sb + (r0 + k) * rs;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = ln + 32 * q;
                        if (j < m)
                            dst[j] = v[k][q];
                    }
                }
            }
        }
        __syncthreads();

        const size_t tile = rel / kTile;
        const int lane0 = (int)((rel % kTile) / 32);
        uint32_t *packed = reinterpret_cast<uint32_t *>((blockIdx.y ? prefs : preads) + T->mc_poff[lo]);
        uint32_t *nmask = WITH_N ? (blockIdx.y ? nrefs : nreads) + T->mc_poff[lo] : nullptr;
        const uint32_t seen = packdev::pack_transpose<WITH_N, true, kPackLanes>(
            sm, m, rs, tile, lane0, packed, nmask, packdev::rotation_step(rs, kPackLanes), kPackThreads);
        // sm is refilled for the next block after this barrier
        if (WITH_N)
            __syncthreads();
        else if (__syncthreads_or(packdev::has_n_bytes(seen)) && threadIdx.x == 0)
            g_batch_unmasked_n = 1u;
    }
}

// The same pack as a persistent, double-buffered kernel for rows that start on
// 16-byte boundaries: each CTA walks blocks blockIdx.x, +gridDim.x, ...; the
// 16-byte chunks of the next block's rows are copied global -> shared with
// cp.async while the current block is transposed, so the gathers' memory
// latency overlaps the transposition.  Padding slots are zero-filled by the
// copy itself (source size 0).
using packdev::cp_async16;
using packdev::cp_async_commit;
using packdev::cp_async_wait;

struct PackBlock {
    int m, rs;
    uint32_t slot0, rel, mc;
};

// Rows left free after each lane's 32 staged rows of length m in the
// persistent pack: with them the lanes of a warp read distinct banks with the
// rows in order (pack_transpose_spaced).  They are used only where a buffer
// of buf_bytes holds them; otherwise (0) the rows are staged densely and
// read in a rotated order (pack_transpose).
__host__ __device__ inline int lane_gap(int m, int buf_bytes)
{
    const int gap = packdev::rotation_step(row_stride(m), kPackLanes);
    const int fits = (kPackSeqs + (kPackLanes - 1) * gap) * row_stride(m) + 16 <= buf_bytes;
    return fits ? gap : 0;
}

// m-class tables of a run, copied to shared memory by the persistent pack.
struct McCache {
    uint32_t n_mc, total;
    uint32_t block[kMaxM + 1], slot[kMaxM];
    uint16_t m[kMaxM];
    uint64_t poff[kMaxM];
    // rows left free after each lane's 32 staged rows (0: rows staged densely
    // and read in a rotated order instead), and that rotation step
    uint8_t gap[kMaxM], rot[kMaxM];
};

__device__ __forceinline__ PackBlock locate_block(const McCache &c, uint32_t blk)
{
    uint32_t lo = 0, hi = c.n_mc;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (c.block[mid] <= blk)
            lo = mid;
        else
            hi = mid;
    }
    PackBlock b;
    b.mc = lo;
    b.m = (int)c.m[lo];
    b.rs = row_stride(b.m);
    b.rel = (blk - c.block[lo]) * kPackSeqs;
    b.slot0 = c.slot[lo] + b.rel;
    return b;
}

// Pipeline of one CTA over its blocks k = 0, 1, 2, ... (block ids blockIdx.x +
// k * gridDim.x): in step k it loads the permutation entries of block k+2
// (one per thread, kept in a register until the end of the step), issues the
// cp.async copies of block k+1's rows (whose permutation entries arrived one
// step earlier), waits for block k's copies and transposes block k.
template <bool WITH_N>
__global__ void __launch_bounds__(kPackThreads)
pack_async_kernel(const Args *__restrict__ a, const Tables *__restrict__ T, int max_m, int buf_bytes,
                  const uint32_t *__restrict__ perm, uint2 *__restrict__ preads,
                  uint2 *__restrict__ prefs, uint32_t *__restrict__ nreads,
                  uint32_t *__restrict__ nrefs)
{
    extern __shared__ __align__(16) uint32_t smw[];
    __shared__ McCache mc;
    __shared__ uint32_t P[3][kPackSeqs];   // permutation entries of three blocks
    const uint8_t *seqs = blockIdx.y ? a->refs : a->reads;
    const uint64_t stride = a->stride;
    if (!rows_on_16_bytes(seqs, stride, max_m) || (blockIdx.y && a->ref_off))
        return;  // pack_kernel does this side
    if (threadIdx.x == 0) {
        mc.n_mc = T->n_mc;
        mc.total = mc.n_mc ? T->mc_block[mc.n_mc] : 0u;
    }
    __syncthreads();
    const uint32_t nmc = mc.n_mc, total = mc.total;
    if (blockIdx.x >= total)
        return;
    for (uint32_t i = threadIdx.x; i <= nmc; i += kPackThreads)
        mc.block[i] = T->mc_block[i];
    for (uint32_t i = threadIdx.x; i < nmc; i += kPackThreads) {
        mc.m[i] = T->mc_m[i];
        mc.slot[i] = T->mc_slot[i];
        mc.poff[i] = T->mc_poff[i];
        mc.gap[i] = (uint8_t)lane_gap((int)T->mc_m[i], buf_bytes);
        mc.rot[i] = (uint8_t)packdev::rotation_step(row_stride((int)T->mc_m[i]), kPackLanes);
    }
    __syncthreads();

    uint8_t *buf0 = reinterpret_cast<uint8_t *>(smw);
    uint8_t *buf1 = buf0 + buf_bytes;
    auto blk_of = [&](uint32_t k) { return blockIdx.x + k * gridDim.x; };
    auto perm_entry = [&](uint32_t k) -> uint32_t {
        const uint32_t blk = blk_of(k);
        if (blk >= total)
            return kNoPair;
        return perm[locate_block(mc, blk).slot0 + threadIdx.x];
    };
    auto issue = [&](uint32_t k, uint8_t *dst) {
        const uint32_t blk = blk_of(k);
        if (blk < total) {
            const PackBlock b = locate_block(mc, blk);
            const int nck = (b.m + 15) >> 4;
            const int gap = mc.gap[b.mc];
            const uint32_t *pk = P[k % 3];
            for (int it = threadIdx.x; it < kPackSeqs * nck; it += kPackThreads) {
                const int r = it / nck, c = it - r * nck;
                const uint32_t pair = pk[r];
                const bool ok = pair != kNoPair;
                const uint8_t *src = ok ? seqs + (uint64_t)pair * stride + 16 * c : seqs;
                // row r of lane r / 32 goes to staged row r + (r / 32) * gap
                cp_async16(dst + (r + (r >> 5) * gap) * b.rs + 16 * c, src, ok ? 16u : 0u);
            }
        }
        cp_async_commit();  // an empty group past the last block keeps the count regular
    };

    // prologue: permutation of blocks 0 and 1, copies of block 0
    P[0][threadIdx.x] = perm_entry(0);
    P[1][threadIdx.x] = perm_entry(1);
    __syncthreads();
    issue(0, buf0);
    for (uint32_t k = 0; blk_of(k) < total; ++k) {
        const uint32_t ahead = perm_entry(k + 2);   // consumed in step k+1
        issue(k + 1, (k & 1) ? buf0 : buf1);
        cp_async_wait<1>();                        // block k's copies are in
        __syncthreads();
        const PackBlock b = locate_block(mc, blk_of(k));
        const size_t tile = b.rel / kTile;
        const int lane0 = (int)((b.rel % kTile) / 32);
        uint32_t *packed = reinterpret_cast<uint32_t *>((blockIdx.y ? prefs : preads) + mc.poff[b.mc]);
        uint32_t *nmask = WITH_N ? (blockIdx.y ? nrefs : nreads) + mc.poff[b.mc] : nullptr;
        const uint32_t *sbuf = reinterpret_cast<const uint32_t *>((k & 1) ? buf1 : buf0);
        const uint32_t seen =
            mc.gap[b.mc] ? packdev::pack_transpose_spaced<WITH_N, kPackLanes>(
                               sbuf, b.m, b.rs, mc.gap[b.mc], tile, lane0, packed, nmask,
                               kPackThreads, (int)threadIdx.x)
                         : packdev::pack_transpose<WITH_N, true, kPackLanes>(
                               sbuf, b.m, b.rs, tile, lane0, packed, nmask, mc.rot[b.mc],
                               kPackThreads);
        P[(k + 2) % 3][threadIdx.x] = ahead;
        // the buffer of block k is refilled in step k+1, after this barrier
        if (WITH_N)
            __syncthreads();
        else if (__syncthreads_or(packdev::has_n_bytes(seen)) && threadIdx.x == 0)
            g_batch_unmasked_n = 1u;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- finalize
__global__ void __launch_bounds__(256)
finalize_kernel(const Args *__restrict__ a, const Tables *__restrict__ T,
                const uint16_t *__restrict__ keys, const uint32_t *__restrict__ ranks,
                const uint8_t *__restrict__ count_slot)
{
    const uint64_t n = a->n;
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((i & ~(uint64_t)31) >= n)
        return;
    uint32_t c = 0xFFu;
    bool acc = false;
    if (i < n) {
        const uint16_t k = keys[i];
        if (k != kBadKey) {
            c = count_slot[T->bin_slot[k] + ranks[i]];
            acc = c <= (uint32_t)(k & (kMaxE - 1));
        }
        if (a->count)
            a->count[i] = (uint8_t)c;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, acc);
    if ((threadIdx.x & 31) == 0)
        a->accept[i >> 5] = word;
}

}  // namespace
}  // namespace batch

cudaError_t take_batch_unmasked_n(uint32_t *seen)
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, batch::g_batch_unmasked_n, sizeof v);
    if (e == cudaSuccess && v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(batch::g_batch_unmasked_n, &zero, sizeof zero);
    }
    *seen = v;
    return e;
}

}  // namespace shouji

using namespace shouji;
using namespace shouji::batch;

// Argument blocks (and captured graphs) a batch object cycles through.
constexpr int kArgBufs = 2;

struct shouji_batch {
    int device = 0;
    int sms = 0;
    size_t max_pairs = 0;
    uint32_t max_m = 0;
    int e_lo = 0, e_hi = 0, with_n = 0;
    size_t slots_cap = 0;
    size_t pack_blocks_cap = 0;
    int pack_grid = 0;      // CTAs per side of the fallback pack (walks the blocks)
    int async_grid = 0;     // CTAs per side of the persistent pack (0: not used)
    int async_buf = 0;      // bytes of one shared-memory buffer
    Args *d_args = nullptr;
    Args *h_args = nullptr;          // kArgBufs pinned argument blocks
    uint32_t *d_hist = nullptr;
    Tables *d_tables = nullptr;
    uint16_t *d_keys = nullptr;
    uint32_t *d_ranks = nullptr, *d_perm = nullptr;
    uint8_t *d_count_slot = nullptr;
    uint2 *d_pr = nullptr, *d_pt = nullptr;
    uint32_t *d_nr = nullptr, *d_nt = nullptr;
    int threads[kMaxE], ctas_per_sm[kMaxE], schedule[kMaxE], u[kMaxE];
    // One graph per argument block: graph k copies block k, so a run waits
    // only for the run kArgBufs runs before it to have started.
    cudaGraph_t graph[kArgBufs] = {};
    cudaGraphExec_t exec[kArgBufs] = {};
    cudaEvent_t done[kArgBufs] = {};
    bool launched[kArgBufs] = {};
    int next = 0;                    // argument block of the next run
    int last = -1;                   // argument block of the last run
    cudaStream_t capture = nullptr;  // private stream the graph is captured on
    cudaStream_t aux[kMaxE] = {};    // graph branches: one per threshold
    cudaEvent_t fork = nullptr, join[kMaxE] = {};
    // Timing events recorded by the graph itself (shouji_batch_timing).
    cudaEvent_t t_begin = nullptr, t_bucketed = nullptr, t_packed = nullptr,
                t_joined = nullptr, t_end = nullptr;
    cudaEvent_t t_e0[kMaxE] = {}, t_e1[kMaxE] = {};
};

namespace {

// An event record that becomes a node of the graph being captured, so its
// time stamp is taken every time the graph runs.
cudaError_t stamp(cudaEvent_t ev, cudaStream_t s)
{
    return ev ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaSuccess;
}

using BatchLaunch = cudaError_t (*)(const FilterParams &, int, int, cudaStream_t);
constexpr BatchLaunch kBatchFilter[kMaxE] = {
    &launch_filter_E<0>,  &launch_filter_E<1>,  &launch_filter_E<2>,  &launch_filter_E<3>,
    &launch_filter_E<4>,  &launch_filter_E<5>,  &launch_filter_E<6>,  &launch_filter_E<7>,
    &launch_filter_E<8>,  &launch_filter_E<9>,  &launch_filter_E<10>, &launch_filter_E<11>,
    &launch_filter_E<12>, &launch_filter_E<13>, &launch_filter_E<14>, &launch_filter_E<15>,
    &launch_filter_E<16>, &launch_filter_E<17>, &launch_filter_E<18>, &launch_filter_E<19>,
    &launch_filter_E<20>, &launch_filter_E<21>, &launch_filter_E<22>, &launch_filter_E<23>,
    &launch_filter_E<24>, &launch_filter_E<25>, &launch_filter_E<26>, &launch_filter_E<27>,
    &launch_filter_E<28>, &launch_filter_E<29>, &launch_filter_E<30>, &launch_filter_E<31>,
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess)
            prev = -1;
        if (prev != dev)
            cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

size_t pack_smem(uint32_t max_m)
{
    size_t best = 0;
    for (uint32_t m = 1; m <= max_m; ++m) {
        const size_t b = (size_t)kPackSeqs * row_stride((int)m) + 16;
        best = b > best ? b : best;
    }
    return best;
}

// Bytes of one buffer of the persistent pack that stages every length up to
// max_m with its lane gaps.
size_t async_smem_spaced(uint32_t max_m)
{
    size_t best = 0;
    for (uint32_t m = 1; m <= max_m; ++m) {
        const size_t b = (size_t)(kPackSeqs + (kPackLanes - 1) *
                                  packdev::rotation_step(row_stride((int)m), kPackLanes)) *
                             row_stride((int)m) + 16;
        best = b > best ? b : best;
    }
    return (best + 15) / 16 * 16;
}

FilterParams filter_params(const shouji_batch *b)
{
    FilterParams p;
    p.tables = b->d_tables;
    p.preads = b->d_pr;
    p.prefs = b->d_pt;
    p.nreads = b->with_n ? b->d_nr : nullptr;
    p.nrefs = b->with_n ? b->d_nt : nullptr;
    p.count_slot = b->d_count_slot;
    p.work = b->d_tables->work;
    p.schedule = 0;
    p.u = 4;
    return p;
}

// The stages before the per-threshold filters, with argument block k.
// `timed`: record the graph's timing events (only inside a capture).
cudaError_t enqueue_prologue(shouji_batch *b, cudaStream_t s, int k, bool timed)
{
    cudaError_t e;
    if (timed && (e = stamp(b->t_begin, s)))
        return e;
    if ((e = cudaMemcpyAsync(b->d_args, b->h_args + k, sizeof(Args), cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = cudaMemsetAsync(b->d_hist, 0, sizeof(uint32_t) * kBins, s)))
        return e;
    if ((e = cudaMemsetAsync(&b->d_tables->n_invalid, 0, sizeof(uint32_t), s)))
        return e;
    if ((e = cudaMemsetAsync(b->d_tables->work, 0, sizeof(uint32_t) * kMaxE, s)))
        return e;
    // a persistent grid: each CTA walks chunks of kClsPairs pairs
    const size_t cls_chunks = (b->max_pairs + kClsPairs - 1) / kClsPairs;
    const size_t cls_cap = (size_t)b->sms * kClsCtasPerSm;
    const unsigned cls_blocks = (unsigned)(cls_chunks < cls_cap ? cls_chunks : cls_cap);
    classify_kernel<<<cls_blocks ? cls_blocks : 1, kClsThreads, 0, s>>>(
        b->d_args, (int)b->max_m, b->e_lo, b->e_hi, b->d_hist, b->d_tables, b->d_keys, b->d_ranks);
    scan_kernel<<<1, 256, 0, s>>>(b->d_hist, b->d_tables);
    fill_kernel<<<b->sms * 4, 256, 0, s>>>(b->d_tables, b->d_perm);
    scatter_kernel<<<b->sms * 8, 256, 0, s>>>(b->d_args, b->d_tables, b->d_keys, b->d_ranks,
                                              b->d_perm);
    if (timed && (e = stamp(b->t_bucketed, s)))
        return e;
    // The persistent double-buffered pack needs rows on 16-byte boundaries;
    // the stride is known only per run, so both forms are in the graph and
    // each exits at once when the other one applies.
    const dim3 pgrid((unsigned)b->pack_grid, 2);
    const dim3 agrid((unsigned)b->async_grid, 2);
    if (b->with_n) {
        pack_kernel<true><<<pgrid, kPackThreads, pack_smem(b->max_m), s>>>(
            b->d_args, b->d_tables, (int)b->max_m, b->d_perm, b->d_pr, b->d_pt, b->d_nr, b->d_nt);
        pack_async_kernel<true><<<agrid, kPackThreads, 2 * b->async_buf, s>>>(
            b->d_args, b->d_tables, (int)b->max_m, b->async_buf, b->d_perm, b->d_pr, b->d_pt,
            b->d_nr, b->d_nt);
    } else {
        pack_kernel<false><<<pgrid, kPackThreads, pack_smem(b->max_m), s>>>(
            b->d_args, b->d_tables, (int)b->max_m, b->d_perm, b->d_pr, b->d_pt, nullptr, nullptr);
        pack_async_kernel<false><<<agrid, kPackThreads, 2 * b->async_buf, s>>>(
            b->d_args, b->d_tables, (int)b->max_m, b->async_buf, b->d_perm, b->d_pr, b->d_pt,
            nullptr, nullptr);
    }
    if ((e = cudaGetLastError()))
        return e;
    return timed ? stamp(b->t_packed, s) : cudaSuccess;
}

cudaError_t enqueue_filter(shouji_batch *b, int E, int threads, int ctas_per_sm, int schedule,
                           int u, cudaStream_t s)
{
    FilterParams p = filter_params(b);
    p.schedule = schedule;
    p.u = u;
    return kBatchFilter[E](p, threads, ctas_per_sm * b->sms, s);
}

// The threshold kernels are independent: in the graph they are parallel
// branches (fork after the pack, join before the finalize), so batches whose
// thresholds each hold little work still fill the GPU.
cudaError_t enqueue_all(shouji_batch *b, cudaStream_t s, int k)
{
    cudaError_t e = enqueue_prologue(b, s, k, true);
    if (e)
        return e;
    if ((e = cudaEventRecord(b->fork, s)))
        return e;
    for (int E = b->e_lo; E <= b->e_hi; ++E) {
        cudaStream_t t = b->aux[E];
        if ((e = cudaStreamWaitEvent(t, b->fork, 0)))
            return e;
        if ((e = stamp(b->t_e0[E], t)))
            return e;
        if ((e = enqueue_filter(b, E, b->threads[E], b->ctas_per_sm[E], b->schedule[E], b->u[E],
                                t)))
            return e;
        if ((e = stamp(b->t_e1[E], t)))
            return e;
        if ((e = cudaEventRecord(b->join[E], t)))
            return e;
        if ((e = cudaStreamWaitEvent(s, b->join[E], 0)))
            return e;
    }
    if ((e = stamp(b->t_joined, s)))
        return e;
    const unsigned fin_blocks = (unsigned)((b->max_pairs + 255) / 256);
    finalize_kernel<<<fin_blocks ? fin_blocks : 1, 256, 0, s>>>(b->d_args, b->d_tables, b->d_keys,
                                                                b->d_ranks, b->d_count_slot);
    if ((e = cudaGetLastError()))
        return e;
    return stamp(b->t_end, s);
}

// Waits for every run still in flight, then drops the graphs.
void drop_graphs(shouji_batch *b)
{
    for (int k = 0; k < kArgBufs; ++k) {
        if (b->launched[k])
            cudaEventSynchronize(b->done[k]);
        b->launched[k] = false;
        if (b->exec[k])
            cudaGraphExecDestroy(b->exec[k]);
        if (b->graph[k])
            cudaGraphDestroy(b->graph[k]);
        b->exec[k] = nullptr;
        b->graph[k] = nullptr;
    }
    b->last = -1;
}

cudaError_t build_graph(shouji_batch *b, cudaStream_t s, int k)
{
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e)
        return e;
    cudaError_t e2 = enqueue_all(b, s, k);
    e = cudaStreamEndCapture(s, &b->graph[k]);
    if (e2)
        return e2;
    if (e)
        return e;
    return cudaGraphInstantiate(&b->exec[k], b->graph[k], 0);
}

void release(shouji_batch *b)
{
    if (!b)
        return;
    DeviceGuard g(b->device);
    drop_graphs(b);
    for (int k = 0; k < kArgBufs; ++k)
        if (b->done[k])
            cudaEventDestroy(b->done[k]);
    for (cudaEvent_t ev : {b->t_begin, b->t_bucketed, b->t_packed, b->t_joined, b->t_end})
        if (ev)
            cudaEventDestroy(ev);
    for (int E = 0; E < kMaxE; ++E) {
        if (b->t_e0[E])
            cudaEventDestroy(b->t_e0[E]);
        if (b->t_e1[E])
            cudaEventDestroy(b->t_e1[E]);
    }
    if (b->capture)
        cudaStreamDestroy(b->capture);
    for (int E = 0; E < kMaxE; ++E) {
        if (b->aux[E])
            cudaStreamDestroy(b->aux[E]);
        if (b->join[E])
            cudaEventDestroy(b->join[E]);
    }
    if (b->fork)
        cudaEventDestroy(b->fork);
    cudaFree(b->d_args);
    if (b->h_args)
        cudaFreeHost(b->h_args);
    cudaFree(b->d_hist);
    cudaFree(b->d_tables);
    cudaFree(b->d_keys);
    cudaFree(b->d_ranks);
    cudaFree(b->d_perm);
    cudaFree(b->d_count_slot);
    cudaFree(b->d_pr);
    cudaFree(b->d_pt);
    cudaFree(b->d_nr);
    cudaFree(b->d_nt);
    delete b;
}

void device_name(char *out, size_t cap, int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
        snprintf(out, cap, "unknown");
        return;
    }
    snprintf(out, cap, "%s", p.name);
    for (char *c = out; *c; ++c)
        if (*c == ' ')
            *c = '_';
}

// Slots a batch of up to n pairs can occupy: every non-empty bucket pads to
// 32 slots and every non-empty m-class to a 1024-slot tile, and there are at
// most min(n, lengths x thresholds) buckets and min(n, lengths) m-classes.
size_t slots_capacity(size_t n, uint32_t max_m, int e_min, int e_max)
{
    const size_t buckets = (size_t)max_m * (size_t)(e_max - e_min + 1);
    const size_t classes = max_m;
    const size_t s = n + 31 * (n < buckets ? n : buckets) + (kTile - 1) * (n < classes ? n : classes);
    return (s + kTile - 1) / kTile * kTile;
}

// Device bytes shouji_batch_create allocates (its cudaMalloc calls, in order).
size_t batch_bytes(size_t max_pairs, uint32_t max_m, int e_min, int e_max, int with_n)
{
    const size_t slots = slots_capacity(max_pairs, max_m, e_min, e_max);
    const size_t packed_u2 = slots / kTile * max_m * kLanes;
    size_t b = sizeof(Args) + sizeof(uint32_t) * kBins + sizeof(Tables) +
               sizeof(uint16_t) * max_pairs + sizeof(uint32_t) * max_pairs +
               sizeof(uint32_t) * slots + slots + 2 * sizeof(uint2) * packed_u2;
    if (with_n)
        b += 2 * sizeof(uint32_t) * packed_u2;
    return b;
}

// Tuning cache: lines "<gpu> <E> <threads> <ctas_per_sm> <schedule> <U> <ms>".
void load_cache(shouji_batch *b, const char *path)
{
    if (!path)
        return;
    FILE *f = fopen(path, "r");
    if (!f)
        return;
    char gpu[128], want[128];
    device_name(want, sizeof(want), b->device);
    int E, th, cps, sch, u;
    double ms;
    while (fscanf(f, "%127s %d %d %d %d %d %lf", gpu, &E, &th, &cps, &sch, &u, &ms) == 7) {
        if (strcmp(gpu, want) == 0 && E >= 0 && E < kMaxE && (th == 64 || th == 128) &&
            cps >= 1 && cps <= 8 && sch >= 0 && sch <= 2 && (u == 4 || (u == 8 && E <= kMaxE8))) {
            b->threads[E] = th;
            b->ctas_per_sm[E] = cps;
            b->schedule[E] = sch;
            b->u[E] = u;
        }
    }
    fclose(f);
}

// Writes argument block k (that of the next run).
shouji_status set_args(shouji_batch *b, int k, const uint8_t *reads, const uint8_t *refs,
                       uint64_t stride, const uint16_t *lens, const uint8_t *E_per_pair,
                       size_t n, uint32_t *accept, uint8_t *count,
                       const uint64_t *ref_off = nullptr)
{
    if (b->launched[k]) {
        // the run that last used block k must have copied it
        cudaError_t e = cudaEventSynchronize(b->done[k]);
        if (e)
            return cuda_status(e);
    }
    Args *a = b->h_args + k;
    a->reads = reads;
    a->refs = refs;
    a->stride = stride;
    a->ref_off = ref_off;
    a->lens = lens;
    a->E_per_pair = E_per_pair;
    a->n = n;
    a->accept = accept;
    a->count = count;
    return SHOUJI_OK;
}

}  // namespace

extern "C" {

size_t shouji_batch_device_bytes(size_t max_pairs, uint32_t max_m, int e_min, int e_max,
                                 int with_n)
{
    if (max_pairs == 0 || max_m < 1 || max_m > SHOUJI_MAX_M || e_min < 0 || e_max > SHOUJI_MAX_E ||
        e_min > e_max)
        return 0;
    return batch_bytes(max_pairs, max_m, e_min, e_max, with_n);
}

shouji_status shouji_batch_create(size_t max_pairs, uint32_t max_m, int e_min, int e_max,
                                  int with_n, const char *tune_cache, shouji_batch **out)
{
    if (!out || max_pairs == 0 || max_pairs >= ((size_t)1 << 31) || max_m < 1 ||
        max_m > SHOUJI_MAX_M || e_min < 0 || e_max > SHOUJI_MAX_E || e_min > e_max)
        return SHOUJI_EINVAL;
    *out = nullptr;
    shouji_batch *b = new (std::nothrow) shouji_batch;
    if (!b)
        return SHOUJI_ENOMEM;
    cudaError_t e = cudaGetDevice(&b->device);
    if (!e)
        e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e) {
        delete b;
        return cuda_status(e);
    }
    b->max_pairs = max_pairs;
    b->max_m = max_m;
    b->e_lo = e_min;
    b->e_hi = e_max;
    b->with_n = with_n ? 1 : 0;
    for (int E = 0; E < kMaxE; ++E) {
        b->threads[E] = 128;
        b->ctas_per_sm[E] = 4;
        b->schedule[E] = 0;
        b->u[E] = 4;
    }
    b->slots_cap = slots_capacity(max_pairs, max_m, e_min, e_max);
    b->pack_blocks_cap = b->slots_cap / kPackSeqs;
    b->pack_grid = (int)(b->pack_blocks_cap < (size_t)b->sms * 8 ? b->pack_blocks_cap
                                                                  : (size_t)b->sms * 8);
    if (b->pack_grid < 1)
        b->pack_grid = 1;
    const size_t packed_u2 = b->slots_cap / kTile * max_m * kLanes;  // uint2 per side
    bool ok = true;
    ok = ok && cudaMalloc(&b->d_args, sizeof(Args)) == cudaSuccess;
    ok = ok && cudaMallocHost(&b->h_args, kArgBufs * sizeof(Args)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_hist, sizeof(uint32_t) * kBins) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_tables, sizeof(Tables)) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_keys, sizeof(uint16_t) * max_pairs) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_ranks, sizeof(uint32_t) * max_pairs) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_perm, sizeof(uint32_t) * b->slots_cap) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_count_slot, b->slots_cap) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_pr, sizeof(uint2) * packed_u2) == cudaSuccess;
    ok = ok && cudaMalloc(&b->d_pt, sizeof(uint2) * packed_u2) == cudaSuccess;
    if (b->with_n) {
        ok = ok && cudaMalloc(&b->d_nr, sizeof(uint32_t) * packed_u2) == cudaSuccess;
        ok = ok && cudaMalloc(&b->d_nt, sizeof(uint32_t) * packed_u2) == cudaSuccess;
    }
    for (int k = 0; k < kArgBufs; ++k)
        ok = ok && cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming) == cudaSuccess;
    for (cudaEvent_t *ev : {&b->t_begin, &b->t_bucketed, &b->t_packed, &b->t_joined, &b->t_end})
        ok = ok && cudaEventCreate(ev) == cudaSuccess;
    for (int E = e_min; E <= e_max && ok; ++E)
        ok = cudaEventCreate(&b->t_e0[E]) == cudaSuccess && cudaEventCreate(&b->t_e1[E]) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int E = e_min; E <= e_max && ok; ++E) {
        ok = cudaStreamCreateWithFlags(&b->aux[E], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[E], cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok) {
        cudaFuncSetAttribute(pack_kernel<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute(pack_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    }
    if (ok) {
        // persistent pack: buffers that hold every length with its lane gaps
        // while at least 3 CTAs fit on an SM, else buffers of dense rows
        // (the lengths whose gaps do not fit are read in a rotated order);
        // as many CTAs per side as fit on the GPU at once
        const size_t dense = (pack_smem(max_m) + 15) / 16 * 16;
        const size_t spaced = async_smem_spaced(max_m);
        auto fit = [&](size_t buf, int *per_sm) -> bool {
            const size_t asmem = 2 * buf;
            bool good = cudaFuncSetAttribute(pack_async_kernel<true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)asmem) == cudaSuccess &&
                        cudaFuncSetAttribute(pack_async_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)asmem) == cudaSuccess;
            cudaFuncSetAttribute(pack_async_kernel<true>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
            cudaFuncSetAttribute(pack_async_kernel<false>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
            *per_sm = 0;
            return good && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                               per_sm, with_n ? pack_async_kernel<true> : pack_async_kernel<false>,
                               kPackThreads, asmem) == cudaSuccess;
        };
        int per_sm = 0;
        b->async_buf = (int)spaced;
        ok = fit(spaced, &per_sm);
        if (!ok || per_sm < 3) {
            cudaGetLastError();
            b->async_buf = (int)dense;
            ok = fit(dense, &per_sm);
        }
        b->async_grid = per_sm > 1 ? per_sm * b->sms / 2 : b->sms;
    }
    if (ok && pack_smem(max_m) > 48 * 1024) {
        ok = cudaFuncSetAttribute(pack_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pack_smem(max_m)) == cudaSuccess &&
             cudaFuncSetAttribute(pack_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pack_smem(max_m)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        release(b);
        return SHOUJI_ENOMEM;
    }
    memset(b->h_args, 0, kArgBufs * sizeof(Args));
    load_cache(b, tune_cache);
    *out = b;
    return SHOUJI_OK;
}

void shouji_batch_destroy(shouji_batch *b) { release(b); }

}  // extern "C"

namespace {

shouji_status batch_run(shouji_batch *b, const uint8_t *reads, const uint8_t *refs,
                        uint64_t stride, const uint64_t *ref_off, const uint16_t *lens,
                        const uint8_t *E_per_pair, size_t n_pairs, uint32_t *out_accept,
                        uint8_t *out_count, void *stream)
{
    if (!b || n_pairs > b->max_pairs || stride < 1)
        return SHOUJI_EINVAL;
    if (n_pairs == 0)
        return SHOUJI_OK;
    if (!reads || !refs || !lens || !E_per_pair || !out_accept)
        return SHOUJI_EINVAL;
    DeviceGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int k = b->next;
    shouji_status st = set_args(b, k, reads, refs, stride, lens, E_per_pair, n_pairs, out_accept,
                                out_count, ref_off);
    if (st)
        return st;
    cudaError_t e = cudaSuccess;
    // The graphs are captured on the object's own stream (the caller's may be
    // the legacy default stream, which cannot be captured) and launched on
    // the caller's.
    if (!b->exec[k] && (e = build_graph(b, b->capture, k)))
        return cuda_status(e);
    if ((e = cudaGraphLaunch(b->exec[k], s)))
        return cuda_status(e);
    if ((e = cudaEventRecord(b->done[k], s)))
        return cuda_status(e);
    b->launched[k] = true;
    b->last = k;
    b->next = (k + 1) % kArgBufs;
    return SHOUJI_OK;
}

}  // namespace

extern "C" {

shouji_status shouji_batch_run(shouji_batch *b, const uint8_t *reads, const uint8_t *refs,
                               uint64_t stride, const uint16_t *lens, const uint8_t *E_per_pair,
                               size_t n_pairs, uint32_t *out_accept, uint8_t *out_count,
                               void *stream)
{
    return batch_run(b, reads, refs, stride, nullptr, lens, E_per_pair, n_pairs, out_accept,
                     out_count, stream);
}

shouji_status shouji_batch_run_at(shouji_batch *b, const uint8_t *reads, uint64_t stride,
                                  const uint8_t *ref_text, const uint64_t *ref_offsets,
                                  const uint16_t *lens, const uint8_t *E_per_pair,
                                  size_t n_pairs, uint32_t *out_accept, uint8_t *out_count,
                                  void *stream)
{
    if (!ref_offsets && n_pairs)
        return SHOUJI_EINVAL;
    return batch_run(b, reads, ref_text, stride, ref_offsets, lens, E_per_pair, n_pairs,
                     out_accept, out_count, stream);
}

shouji_status shouji_batch_shape(shouji_batch *b, int E, int *threads, int *ctas_per_sm,
                                 int *schedule, int *windows)
{
    if (!b || E < 0 || E >= kMaxE || !threads || !ctas_per_sm || !schedule || !windows)
        return SHOUJI_EINVAL;
    *threads = b->threads[E];
    *ctas_per_sm = b->ctas_per_sm[E];
    *schedule = b->schedule[E];
    *windows = b->u[E];
    return SHOUJI_OK;
}

shouji_status shouji_batch_timing(shouji_batch *b, float *ms, int n)
{
    if (!b || !ms || n < SHOUJI_BATCH_TIMES)
        return SHOUJI_EINVAL;
    for (int i = 0; i < SHOUJI_BATCH_TIMES; ++i)
        ms[i] = -1.f;
    if (b->last < 0)
        return SHOUJI_OK;
    DeviceGuard g(b->device);
    cudaError_t e = cudaEventSynchronize(b->done[b->last]);
    if (e)
        return cuda_status(e);
    auto span = [&](cudaEvent_t a, cudaEvent_t z, float *out) -> cudaError_t {
        return cudaEventElapsedTime(out, a, z);
    };
    if ((e = span(b->t_begin, b->t_end, &ms[0])) || (e = span(b->t_begin, b->t_bucketed, &ms[1])) ||
        (e = span(b->t_bucketed, b->t_packed, &ms[2])) ||
        (e = span(b->t_packed, b->t_joined, &ms[3])) || (e = span(b->t_joined, b->t_end, &ms[4])))
        return cuda_status(e);
    for (int E = b->e_lo; E <= b->e_hi; ++E)
        if ((e = span(b->t_e0[E], b->t_e1[E], &ms[5 + E])))
            return cuda_status(e);
    return SHOUJI_OK;
}

shouji_status shouji_batch_invalid(shouji_batch *b, uint64_t *n_invalid)
{
    if (!b || !n_invalid)
        return SHOUJI_EINVAL;
    DeviceGuard g(b->device);
    cudaError_t e = b->last >= 0 ? cudaEventSynchronize(b->done[b->last]) : cudaSuccess;
    uint32_t v = 0;
    if (!e)
        e = cudaMemcpy(&v, &b->d_tables->n_invalid, sizeof(v), cudaMemcpyDeviceToHost);
    if (e)
        return cuda_status(e);
    *n_invalid = b->last >= 0 ? v : 0;
    return SHOUJI_OK;
}

shouji_status shouji_batch_tune(shouji_batch *b, const uint8_t *reads, const uint8_t *refs,
                                uint64_t stride, const uint16_t *lens, const uint8_t *E_per_pair,
                                size_t n_pairs, uint32_t *out_accept, uint8_t *out_count,
                                const char *tune_cache, void *stream)
{
    if (!b || n_pairs == 0 || n_pairs > b->max_pairs || !reads || !refs || !lens || !E_per_pair ||
        !out_accept)
        return SHOUJI_EINVAL;
    DeviceGuard g(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    drop_graphs(b);  // waits for the runs in flight; re-captured after tuning
    shouji_status st = set_args(b, 0, reads, refs, stride, lens, E_per_pair, n_pairs, out_accept,
                                out_count);
    if (st)
        return st;
    cudaError_t e = enqueue_prologue(b, s, 0, false);
    if (!e)
        e = cudaStreamSynchronize(s);
    if (e)
        return cuda_status(e);
    uint32_t groups[kMaxE];
    if ((e = cudaMemcpy(groups, b->d_tables->ec_groups, sizeof(groups), cudaMemcpyDeviceToHost)))
        return cuda_status(e);
    struct Cand {
        int th, cps, sch, u;
    };
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    char gpu[128];
    device_name(gpu, sizeof(gpu), b->device);
    FILE *f = tune_cache ? fopen(tune_cache, "a") : nullptr;
    for (int E = b->e_lo; E <= b->e_hi && !e; ++E) {
        if (!groups[E])
            continue;
        // launch shapes x schedules x windows per chunk
        std::vector<Cand> cands;
        for (int u : {4, 8}) {
            if (u == 8 && E > kMaxE8)
                continue;
            for (int sch = 0; sch < 3; ++sch) {
                for (int cps : {1, 2, 3, 4})
                    cands.push_back({128, cps, sch, u});
                for (int cps : {2, 4, 6, 8})
                    cands.push_back({64, cps, sch, u});
            }
        }
        float best = 1e30f;
        Cand pick = {b->threads[E], b->ctas_per_sm[E], b->schedule[E], b->u[E]};
        for (const Cand &c : cands) {
            auto once = [&]() -> cudaError_t {
                cudaError_t r = cudaMemsetAsync(b->d_tables->work, 0, sizeof(uint32_t) * kMaxE, s);
                return r ? r : enqueue_filter(b, E, c.th, c.cps, c.sch, c.u, s);
            };
            if ((e = once()))  // warm-up
                break;
            const int reps = 3;
            float ms_sum = 0.f;
            for (int r = 0; r < reps && !e; ++r) {
                // the counter reset stays outside the timed interval
                if ((e = cudaMemsetAsync(b->d_tables->work, 0, sizeof(uint32_t) * kMaxE, s)))
                    break;
                cudaEventRecord(t0, s);
                if ((e = enqueue_filter(b, E, c.th, c.cps, c.sch, c.u, s)))
                    break;
                cudaEventRecord(t1, s);
                if ((e = cudaEventSynchronize(t1)))
                    break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, t0, t1);
                ms_sum += ms;
            }
            if (e)
                break;
            const float ms = ms_sum / reps;
            if (ms < best) {
                best = ms;
                pick = c;
            }
        }
        if (e)
            break;
        b->threads[E] = pick.th;
        b->ctas_per_sm[E] = pick.cps;
        b->schedule[E] = pick.sch;
        b->u[E] = pick.u;
        if (f)
            fprintf(f, "%s %d %d %d %d %d %.6f\n", gpu, E, pick.th, pick.cps, pick.sch, pick.u,
                    best);
    }
    if (f)
        fclose(f);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (e)
        return cuda_status(e);
    drop_graphs(b);  // re-captured with the tuned shapes on the next run
    return SHOUJI_OK;
}

}  // extern "C"
