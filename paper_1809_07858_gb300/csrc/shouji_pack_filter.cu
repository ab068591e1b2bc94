// shouji_pack_filter: pack of both sequence sets and the Shouji filter
// (arXiv 1809.07858, Sec. 2.2) in one warp-specialized persistent kernel.
//
// The pack is bound by HBM (it reads m bytes of ASCII per sequence) and the
// filter by the integer ALU (it reads 2m/4 packed bytes per pair, from L2
// when they were just written).  Run one after the other, the ALU idles
// through the pack and HBM through the filter.  Here one CTA per SM holds
// both:
//  - 16 producer warps in two independent groups of 8 stream the CTA's range
//    of tiles (1024 pairs each).  A tile is 8 blocks of 256 sequences (4 of
//    reads, then 4 of refs); group g takes the blocks i = g (mod 2).  Each
//    group has its own named barrier and its own ring of shared-memory
//    buffers, filled by bulk copies (one per block, completing on the
//    buffer's mbarrier; the ASCII lines are marked to leave L2 first), so the
//    two groups' transpositions overlap.  A block costs a group about the
//    latency of one transposition item plus two barriers, whatever its size,
//    so two groups double the pack rate.
//  - 8 consumer warps filter the tiles already packed; a consumer that is
//    done with a tile takes the next one from a counter in shared memory, so
//    the tiles go to whichever consumer is free.
// Tiles go through a queue of kSlots (12) slots: tile r of the CTA's range uses
// slot r % kSlots, whose two mbarriers hand it over: `ready` (all 512
// producer threads arrive once their words of the tile are written) and
// `freed` (the consumer's 32 threads arrive once they have filtered it).
// The producers complete tile r only after tile r - kSlots is freed, so at
// most kSlots packed tiles are in flight per CTA (they stay within L2) and a
// slot's phases never run two ahead of a waiter.  With kSlots at least the
// number of consumers, the tile r - kSlots has always been packed when a
// consumer takes tile r (consumers take tiles in order and each holds one),
// so the parity of each phase a consumer waits for is never ambiguous.  A
// slow consumer holds up only its own slot: the producers go on packing the
// next tiles for the others.  The producers wait only on consumer steps that
// depend on phases the producers completed before, so the hand-over cannot
// deadlock; every wait is bounded all the same (about a second), and a wait
// that runs out ends the warps concerned and is counted for
// shouji_wait_failures().
//
// Registers: the CTA is launched with 768 threads at 80 registers (61,440 of
// the SM's 65,536).  The producers give theirs down to 56 and the consumers
// take them up to 128 (setmaxnreg): 512 x 56 + 256 x 128 = 768 x 80, so the
// consumers' request is always met.  The host launches the kernel only when
// its compiled register count is exactly 80.
//
// Outputs are those of shouji_pack on both sets followed by shouji_filter:
// the packed arrays stay in HBM for reuse (e.g. at another threshold).
#include "shouji_internal.cuh"
#include "shouji_pack.cuh"
#include "shouji_filter.cuh"

namespace shouji {
namespace {

using namespace packdev;

constexpr int kConsumers = 8;                      // filter warps per CTA
#ifndef SHOUJI_FUSED_SLOTS
#define SHOUJI_FUSED_SLOTS 12
#endif
constexpr int kSlots = SHOUJI_FUSED_SLOTS;         // tiles in flight per CTA
static_assert(kSlots >= kConsumers, "a consumer's wait needs the slot's previous phase done");
constexpr int kGroups = 2;                         // producer groups
constexpr int kGroupThreads = 256;                 // 8 warps per group
constexpr int kProducers = kGroups * kGroupThreads;
constexpr int kFusedThreads = kConsumers * 32 + kProducers;
constexpr int kLaunchRegs = 80;
constexpr int kProducerRegs = 56;
constexpr int kConsumerRegs = 128;
static_assert(kProducers * kProducerRegs + kConsumers * 32 * kConsumerRegs ==
                  kFusedThreads * kLaunchRegs,
              "the register split must add up to the launch's registers");
static_assert(kFusedThreads * kLaunchRegs <= 65536, "one CTA per SM");
constexpr int kBlockSeqs = 256;                    // sequences per staged block
constexpr int kBlockLanes = kBlockSeqs / 32;       // tile lanes per block
constexpr int kHalfBlocks = kTile / kBlockSeqs;    // blocks per tile and set
constexpr int kBlocksPerTile = 2 * kHalfBlocks;    // reads, then refs
constexpr int kMaxRing = 3;                        // buffers per group
constexpr int kRingBytes = 200 * 1024;             // shared memory for both rings
static_assert(SHOUJI_FUSED_MAX_E == 5, "consumers have 128 registers");

__device__ unsigned int g_fused_wait_failures;
// Set when the producers read an 'N' (the fused kernel has no N masks; see
// shouji_unmasked_n).
__device__ unsigned int g_fused_unmasked_n;

// Named barrier of producer group g (barrier 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "n"(kGroupThreads) : "memory");
}

// Group barrier that also returns whether any thread of the group passed p.
__device__ __forceinline__ bool group_sync_or(int g, bool p)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n"
        " bar.red.or.pred o, %2, %3, q;\n selp.u32 %0, 1, 0, o;\n}\n"
        : "=r"(r) : "r"((uint32_t)p), "r"(1 + g), "n"(kGroupThreads) : "memory");
    return r != 0;
}

struct FusedArgs {
    const uint8_t *reads, *refs;   // n rows of m ASCII bytes each, contiguous
    size_t n;
    int m;
    uint32_t *packed_r, *packed_t; // packed outputs (layout of shouji_pack), or the rings
    int ring_mode;                 // 1: tile t goes to entry blockIdx.x * kSlots + t % kSlots
                                   // of packed_r / packed_t (per-CTA rings, no output)
    uint32_t *accept;
    uint8_t *count;
    int rot_step;
    int ring;                      // buffers per group (2..kMaxRing)
    int buf_bytes;                 // bytes per buffer
};

// Producer group g: blocks i = g, g + 2, g + 4, ... of the CTA's range; the
// group's j-th block goes through buffer j % ring of the group's ring.
// LAYOUT: 0 rows of any length, 1 m % 4 == 0, 2 m % 8 == 4 (odd words per row).
template <int LAYOUT>
__device__ void produce(const FusedArgs &a, uint8_t *ring, uint64_t *full, uint64_t *ready,
                        uint64_t *freed, size_t T0, size_t T1)
{
    const int ptid = (int)threadIdx.x - kConsumers * 32;
    const int g = ptid / kGroupThreads, gtid = ptid % kGroupThreads;
    uint8_t *myring = ring + (size_t)g * a.ring * a.buf_bytes;
    uint64_t *myfull = full + g * kMaxRing;
    const size_t nblk = (T1 - T0) * kBlocksPerTile;
    const size_t njobs = nblk > (size_t)g ? (nblk - g + kGroups - 1) / kGroups : 0;
    // block i: tile T0 + i / kBlocksPerTile; the first kHalfBlocks blocks of
    // a tile are reads, the next ones refs
    auto rows_of = [&](size_t i, size_t &seq0) -> int {
        const size_t t = T0 + i / kBlocksPerTile;
        seq0 = t * kTile + (i % kHalfBlocks) * kBlockSeqs;
        const size_t left = seq0 < a.n ? a.n - seq0 : 0;
        return (int)(left < (size_t)kBlockSeqs ? left : (size_t)kBlockSeqs);
    };
    auto src_of = [&](size_t i, size_t seq0) -> const uint8_t * {
        return ((i / kHalfBlocks) % 2 ? a.refs : a.reads) + seq0 * (size_t)a.m;
    };
    // The ASCII rows are read once: their lines leave L2 first, so that the
    // packed words written for the filter warps stay there until read.
    const uint64_t policy = l2_evict_first_policy();
    auto issue = [&](size_t j) {  // one thread: the group's j-th block
        const size_t i = j * kGroups + g;
        size_t seq0;
        const int rows = rows_of(i, seq0);
        const uint32_t bytes = (uint32_t)(rows * a.m) & ~15u;
        const int b = (int)(j % (size_t)a.ring);
        mbar_arrive_expect_tx(&myfull[b], bytes);
        if (bytes)
            bulk_copy_g2s_hint(myring + (size_t)b * a.buf_bytes, src_of(i, seq0), bytes,
                               &myfull[b], policy);
    };

    size_t issued = 0;  // jobs whose copies have been issued (same in every thread)
    for (; issued < (size_t)(a.ring - 1) && issued < njobs; ++issued)
        if (gtid == 0)
            issue(issued);
    size_t j = 0;        // on failure: the first job whose copy may be in flight
    bool failed = false;
    uint32_t seen = 0;   // OR of the bases this thread read
    for (; j < njobs; ++j) {
        if (issued < njobs) {
            if (gtid == 0) {
                fence_proxy_async_smem();  // that buffer was read in the last round
                issue(issued);
            }
            ++issued;
        }
        const size_t i = j * kGroups + g;
        const int b = (int)(j % (size_t)a.ring);
        const bool ok = mbar_wait_bounded(&myfull[b], (uint32_t)((j / a.ring) & 1));
        size_t seq0;
        const int nbytes = rows_of(i, seq0) * a.m;
        const uint8_t *src = src_of(i, seq0);
        uint8_t *buf = myring + (size_t)b * a.buf_bytes;
        for (int x = (nbytes & ~15) + gtid; x < a.buf_bytes; x += kGroupThreads)
            buf[x] = x < nbytes ? __ldg(src + x) : (uint8_t)0;
        if (group_sync_or(g, !ok)) {
            failed = true;
            break;
        }
        const size_t t = T0 + i / kBlocksPerTile;
        const int slot = (int)((t - T0) % kSlots);
        const size_t k = (t - T0) / kSlots;
        // The producers complete tile t only after tile t - kSlots is freed.
        // In ring mode tile t is written over the ring entry of tile t - kSlots,
        // so the wait comes before the group's first block of t instead of
        // before its last.
        const bool first = i % kBlocksPerTile < kGroups;
        const bool last = i % kBlocksPerTile >= kBlocksPerTile - kGroups;
        if (k > 0 && (a.ring_mode ? first : last)) {
            const bool was_freed = mbar_wait_bounded(&freed[slot], (uint32_t)((k - 1) & 1));
            if (group_sync_or(g, !was_freed)) {
                failed = true;
                ++j;
                break;
            }
        }
        const size_t wt = a.ring_mode ? (size_t)blockIdx.x * kSlots + slot : t;
        uint32_t *dst = (i / kHalfBlocks) % 2 ? a.packed_t : a.packed_r;
        const int lane0 = (int)(i % kHalfBlocks) * kBlockLanes;
        if constexpr (LAYOUT == 2)
            seen |= pack_transpose_w_odd(reinterpret_cast<const uint32_t *>(buf), a.m, wt, lane0,
                                         dst, kGroupThreads, gtid);
        else
            seen |= pack_transpose_by<false, LAYOUT == 1, kBlockLanes>(
                reinterpret_cast<const uint32_t *>(buf), a.m, a.m, wt, lane0, dst, nullptr,
                a.rot_step, kGroupThreads, gtid);
        if (last)
            mbar_arrive(&ready[slot]);  // release: this thread's words of tile t
        group_sync(g);  // buffer b may be refilled
    }
    if (failed) {
        if (gtid == 0) {
            atomicAdd(&g_fused_wait_failures, 1u);
            for (size_t q = j; q < issued; ++q)  // copies that may still be in flight
                mbar_wait_bounded(&myfull[q % a.ring], (uint32_t)((q / a.ring) & 1));
        }
        return;
    }
    // every thread of the group gets here (a failure is seen by the whole group)
    if (group_sync_or(g, has_n_bytes(seen)) && gtid == 0)
        g_fused_unmasked_n = 1u;
}

template <int E>
__device__ void consume(const FusedArgs &a, uint64_t *ready, uint64_t *freed,
                        unsigned int *next_tile, size_t T0, size_t T1)
{
    constexpr int U = SHOUJI_FILTER_U;
    const int lane = (int)threadIdx.x & 31;
    const size_t n_groups = groups_of(a.n);
    const int m = a.m;
    for (;;) {
        unsigned int r = 0;  // the next tile of the range, the same in the whole warp
        if (lane == 0)
            r = atomicAdd(next_tile, 1u);
        r = __shfl_sync(~0u, r, 0);
        const size_t t = T0 + r;
        if (t >= T1)
            break;
        const int slot = (int)(r % kSlots);
        const uint32_t k = r / kSlots;
        const bool ok = mbar_wait_bounded(&ready[slot], k & 1u);
        if (!__all_sync(~0u, ok)) {
            if (lane == 0)
                atomicAdd(&g_fused_wait_failures, 1u);
            return;
        }
        const size_t grp = t * kLanes + lane;  // this thread's group of 32 pairs
        if (grp >= n_groups) {
            mbar_arrive(&freed[slot]);
            continue;
        }
        const size_t wt = a.ring_mode ? (size_t)blockIdx.x * kSlots + slot : t;
        const size_t base = wt * (size_t)m * kLanes + lane;
        filt::View v;
        v.rd = reinterpret_cast<const uint2 *>(a.packed_r) + base;
        v.rf = reinterpret_cast<const uint2 *>(a.packed_t) + base;
        v.rdn = v.rfn = nullptr;
        v.vec = nullptr;
        v.m = m;
        uint32_t inactive[E + 1];
#pragma unroll
        for (int i = 0; i <= E; ++i)
            inactive[i] = 0u;
        uint32_t C[8];
        filt::filter_group<E, U, 0, true>(v, inactive, C);
        uint32_t cw[8];
        filt::counts_to_bytes(C, cw);
        uint32_t acc = filt::le_const<E>(C);
        const size_t first = grp * 32;
        const size_t left = a.n - first;
        if (left < 32)
            acc &= (1u << left) - 1u;
        a.accept[grp] = acc;
        if (a.count) {
            if (left >= 32 && ((uintptr_t)(a.count + first) % 16 == 0)) {
                uint4 *dst = reinterpret_cast<uint4 *>(a.count + first);
                dst[0] = make_uint4(cw[0], cw[1], cw[2], cw[3]);
                dst[1] = make_uint4(cw[4], cw[5], cw[6], cw[7]);
            } else {
                for (int b = 0; b < 32 && (size_t)b < left; ++b)
                    a.count[first + b] = (uint8_t)(cw[b >> 2] >> (8 * (b & 3)));
            }
        }
        mbar_arrive(&freed[slot]);  // done with tile t
    }
}

template <int E, int LAYOUT>
__global__ void __launch_bounds__(kFusedThreads, 1) pack_filter_kernel(FusedArgs a)
{
    extern __shared__ __align__(128) uint8_t ring[];
    __shared__ __align__(8) uint64_t full[kGroups * kMaxRing], ready[kSlots], freed[kSlots];
    __shared__ unsigned int next_tile;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kGroups * kMaxRing; ++b)
            mbar_init(&full[b], 1);
        for (int q = 0; q < kSlots; ++q) {
            mbar_init(&ready[q], kProducers);
            mbar_init(&freed[q], 32);
        }
        next_tile = 0;
        mbar_init_fence();
    }
    __syncthreads();
    // a balanced contiguous range of tiles per CTA (uniform over the CTA)
    const size_t n_tiles = tiles_of(a.n);
    const size_t T0 = n_tiles * blockIdx.x / gridDim.x;
    const size_t T1 = n_tiles * (blockIdx.x + 1) / gridDim.x;
    if (T0 >= T1)
        return;
    // warpgroups 0-1 consume, 2-5 produce
    if (threadIdx.x < kConsumers * 32) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kConsumerRegs));
        consume<E>(a, ready, freed, &next_tile, T0, T1);
    } else {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kProducerRegs));
        produce<LAYOUT>(a, ring, full, ready, freed, T0, T1);
    }
}

// The register split above holds only at exactly kLaunchRegs per thread:
// cudaErrorNotSupported when the compiled kernel has another count.
template <int E, int LAYOUT>
cudaError_t check_regs()
{
    static int regs = -1;
    if (regs < 0) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, pack_filter_kernel<E, LAYOUT>);
        if (e != cudaSuccess)
            return e;
        regs = fa.numRegs;
    }
    return regs == kLaunchRegs ? cudaSuccess : cudaErrorNotSupported;
}

int layout_of(int m) { return m % 8 == 4 ? 2 : m % 4 == 0 ? 1 : 0; }

template <int E>
cudaError_t check_regs_E(int m)
{
    switch (layout_of(m)) {
    case 2: return check_regs<E, 2>();
    case 1: return check_regs<E, 1>();
    default: return check_regs<E, 0>();
    }
}

template <int E, int LAYOUT>
cudaError_t launch_fused_ta(const FusedArgs &a, cudaStream_t s)
{
    cudaError_t e0 = check_regs<E, LAYOUT>();
    if (e0 != cudaSuccess)
        return e0;
    const size_t smem = (size_t)kGroups * a.ring * a.buf_bytes;
    cudaError_t e = cudaFuncSetAttribute(pack_filter_kernel<E, LAYOUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const unsigned grid = (unsigned)pack_filter_grid(a.n, sms);
    pack_filter_kernel<E, LAYOUT><<<grid, kFusedThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int E>
cudaError_t launch_fused_E(const FusedArgs &a, cudaStream_t s)
{
    if (a.m % 8 == 4)
        return launch_fused_ta<E, 2>(a, s);
    if (a.m % 4 == 0)
        return launch_fused_ta<E, 1>(a, s);
    return launch_fused_ta<E, 0>(a, s);
}

using CheckFn = cudaError_t (*)(int);
constexpr CheckFn kCheck[SHOUJI_FUSED_MAX_E + 1] = {
    &check_regs_E<0>, &check_regs_E<1>, &check_regs_E<2>,
    &check_regs_E<3>, &check_regs_E<4>, &check_regs_E<5>,
};

using FusedFn = cudaError_t (*)(const FusedArgs &, cudaStream_t);
constexpr FusedFn kFused[SHOUJI_FUSED_MAX_E + 1] = {
    &launch_fused_E<0>, &launch_fused_E<1>, &launch_fused_E<2>,
    &launch_fused_E<3>, &launch_fused_E<4>, &launch_fused_E<5>,
};

int ring_for(int m, int &buf_bytes)
{
    // a buffer holds 256 rows and 16 bytes of zero padding, rounded up to 128
    buf_bytes = (kBlockSeqs * m + 16 + 127) / 128 * 128;
    const int fit = kRingBytes / (kGroups * buf_bytes);
    return fit < kMaxRing ? fit : kMaxRing;
}

}  // namespace

bool pack_filter_fusable(int m, int E)
{
    int buf_bytes;
    return E >= 0 && E <= SHOUJI_FUSED_MAX_E && m >= 1 && ring_for(m, buf_bytes) >= 2;
}

cudaError_t pack_filter_kernel_applies(int m, int E, bool *applies)
{
    *applies = false;
    if (!pack_filter_fusable(m, E))
        return cudaSuccess;
    const cudaError_t e = kCheck[E](m);
    if (e == cudaErrorNotSupported)
        return cudaSuccess;
    *applies = e == cudaSuccess;
    return e;
}

size_t pack_filter_grid(size_t n, int sms)
{
    const size_t n_tiles = tiles_of(n);
    return n_tiles < (size_t)sms ? n_tiles : (size_t)sms;
}

size_t pack_filter_ring_words(size_t n, int m, int sms)
{
    return pack_filter_grid(n, sms) * kSlots * (size_t)m * kLanes * 2;
}

cudaError_t launch_pack_filter(const uint8_t *reads, const uint8_t *refs, size_t n, int m, int E,
                               uint32_t *packed_r, uint32_t *packed_t, uint32_t *accept,
                               uint8_t *count, cudaStream_t s, bool ring_mode)
{
    if (!pack_filter_fusable(m, E))
        return cudaErrorNotSupported;
    FusedArgs a;
    a.reads = reads;
    a.refs = refs;
    a.n = n;
    a.m = m;
    a.packed_r = packed_r;
    a.packed_t = packed_t;
    a.ring_mode = ring_mode ? 1 : 0;
    a.accept = accept;
    a.count = count;
    a.rot_step = rotation_step(m, kBlockLanes);
    a.ring = ring_for(m, a.buf_bytes);
    return kFused[E](a, s);
}

cudaError_t take_fused_unmasked_n(uint32_t *seen)
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_fused_unmasked_n, sizeof v);
    if (e == cudaSuccess && v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_fused_unmasked_n, &zero, sizeof zero);
    }
    *seen = v;
    return e;
}

cudaError_t take_fused_wait_failures(uint32_t *count)
{
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_fused_wait_failures, sizeof v);
    if (e == cudaSuccess && v) {
        const unsigned int zero = 0;
        e = cudaMemcpyToSymbol(g_fused_wait_failures, &zero, sizeof zero);
    }
    *count = v;
    return e;
}

}  // namespace shouji
