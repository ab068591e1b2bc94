// Device helpers of shouji_pack, shared with the batched path.
#pragma once

#include "shouji_internal.cuh"

namespace shouji {
namespace packdev {

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

// Packing without an N mask reads an 'N' as 'G' (both have bits 2 and 1
// set).  The packs therefore OR together every staged word they read and
// look at bit 3 of each byte: it is clear in 'A', 'C', 'G' and 'T' and set
// in 'N' (0x4E) and 'n'.  A block in which it is set is counted for
// shouji_unmasked_n(), so that a caller learns that such results differ from
// the ones an N mask gives.
__device__ __forceinline__ bool has_n_bytes(uint32_t seen) { return (seen & 0x08080808u) != 0; }

// Phase 2 of the pack: the staged rows (row r = sequence r of the block, at
// byte r * rs of sm, m bases each) -> the bit-sliced words of lanes
// lane0 .. lane0+LANES-1 of a tile.  A thread owns (lane, 4 consecutive
// positions); a warp covers LANES lanes x 32/LANES position quads.
// ALIGNED: rs % 4 == 0, so every 4-position word of a row is word-aligned.
// The items are shared out among nthreads threads, this one being number tid.
// Without WITH_N, returns the OR of the bases this thread read (bytes past
// the end of a row left out), for has_n_bytes; with it, 0.
template <bool WITH_N, bool ALIGNED, int LANES = 8>
__device__ __forceinline__ uint32_t pack_transpose_by(const uint32_t *__restrict__ sm, int m,
                                                      int rs, size_t tile, int lane0,
                                                      uint32_t *__restrict__ packed,
                                                      uint32_t *__restrict__ nmask, int rot_step,
                                                      int nthreads, int tid)
{
    const int J = (m + 3) >> 2;
    uint32_t seen = 0;
    for (int item = tid; item < LANES * J; item += nthreads) {
        const int l = item % LANES, j = item / LANES;
        const int rot = (rot_step * l) & 31;     // visit sequence (s + rot) % 32 at step s
        // bytes of the item's words that hold bases (the last word of a row
        // may run past its end)
        const uint32_t keep = 4 * j + 4 <= m ? ~0u : (1u << (8 * (m - 4 * j))) - 1u;
        uint32_t yh[4], yl[4], yn[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            uint32_t h = 0, lo = 0, nn = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int s = (8 * t + u + rot) & 31;
                const int o = (32 * l + s) * rs + 4 * j;   // byte offset of the 4 bases
                uint32_t w;
                if (ALIGNED) {
                    w = sm[o >> 2];
                } else {
                    w = __funnelshift_r(sm[o >> 2], sm[(o >> 2) + 1], 8 * (o & 3));
                }
                h |= ((w >> 2) & 0x01010101u) << u;
                lo |= ((w >> 1) & 0x01010101u) << u;
                if (WITH_N)
                    nn |= (n_bytes(w) >> 7) << u;
                else
                    seen |= w & keep;
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
                // bit k of H holds sequence (k + rot) % 32: rotate left by rot
                reinterpret_cast<uint2 *>(packed)[wi] =
                    make_uint2(__funnelshift_l(H[q], H[q], rot), __funnelshift_l(L[q], L[q], rot));
                if (WITH_N)
                    nmask[wi] = __funnelshift_l(N[q], N[q], rot);
            }
        }
    }
    return seen;
}

// pack_transpose_by for 8 lanes of rows with an odd number W = m / 4 of
// words (m % 8 == 4), no N mask.  Lane l visits its 32 sequences in 8 groups
// of 4 consecutive rows, starting at group l: step k = 4q + v reads sequence
// 4((q + l) % 8) + v.  The 8 lanes x 4 position quads of a warp then read 32
// distinct banks (4W * g mod 32 takes 8 distinct values over the 8 groups g
// when W is odd), the row address is found once per 4 words, and each
// base's bits are shifted straight to their place (a left shift where
// possible) and merged with one mask-and-or per plane.  The output words are
// rotated back by 4l, as in pack_transpose_by.  Returns the OR of the words
// read, for has_n_bytes.
__device__ __forceinline__ uint32_t pack_transpose_w_odd(const uint32_t *__restrict__ sm, int m,
                                                         size_t tile, int lane0,
                                                         uint32_t *__restrict__ packed,
                                                         int nthreads, int tid)
{
    constexpr int LANES = 8;
    const int W = m >> 2;
    uint32_t seen = 0;
    for (int item = tid; item < LANES * W; item += nthreads) {
        const int l = item % LANES, j = item / LANES;
        const uint32_t *lane_rows = sm + 32 * l * W + j;  // word j of the lane's first row
        uint32_t yh[4], yl[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            uint32_t h = 0, lo = 0;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const uint32_t *grp = lane_rows + ((2 * t + half + l) & 7) * 4 * W;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int u = 4 * half + v;  // bit of each byte that step 8t + u fills
                    const uint32_t w = grp[v * W];
                    seen |= w;
                    // bit 2 (hi) and bit 1 (lo) of each byte, moved to bit u
                    const uint32_t xh = u >= 2 ? w << (u - 2) : w >> (2 - u);
                    const uint32_t xl = u >= 1 ? w << (u - 1) : w >> 1;
                    h |= xh & (0x01010101u << u);
                    lo |= xl & (0x01010101u << u);
                }
            }
            yh[t] = h;
            yl[t] = lo;
        }
        uint32_t H[4], L[4];
        transpose4x4(yh[0], yh[1], yh[2], yh[3], H);
        transpose4x4(yl[0], yl[1], yl[2], yl[3], L);
        const int rot = 4 * l;  // bit k holds sequence (k + 4l) % 32: rotate left by 4l
        const int lane = lane0 + l;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const size_t wi = (tile * (size_t)m + 4 * j + q) * 32 + lane;
            reinterpret_cast<uint2 *>(packed)[wi] =
                make_uint2(__funnelshift_l(H[q], H[q], rot), __funnelshift_l(L[q], L[q], rot));
        }
    }
    return seen;
}

// pack_transpose_by for staged rows laid out so that no rotation is needed:
// the 32 rows of lane l of the block start at row l * (32 + gap) (a gap of
// `gap` rows after each lane), with gap * (rs / 4) = 32 / LANES (mod 32)
// (rotation_step), so that at every step the LANES lanes of a warp read
// banks 32 / LANES apart.  A thread owns (lane, 4 consecutive positions) and
// reads its lane's rows in order, one pointer step per row, so each base
// costs a shift and a mask-and-or per plane and no address arithmetic; the
// output words need no rotation.  Requires rs % 4 == 0.  Without WITH_N,
// returns the OR of the bases read (bytes past the end of a row left out).
template <bool WITH_N, int LANES>
__device__ __forceinline__ uint32_t pack_transpose_spaced(const uint32_t *__restrict__ sm, int m,
                                                          int rs, int gap, size_t tile,
                                                          int lane0,
                                                          uint32_t *__restrict__ packed,
                                                          uint32_t *__restrict__ nmask,
                                                          int nthreads, int tid)
{
    const int J = (m + 3) >> 2;
    const int ws = rs >> 2;  // words per staged row
    uint32_t seen = 0;
    for (int item = tid; item < LANES * J; item += nthreads) {
        const int l = item % LANES, j = item / LANES;
        const uint32_t keep = 4 * j + 4 <= m ? ~0u : (1u << (8 * (m - 4 * j))) - 1u;
        const uint32_t *row = sm + l * (32 + gap) * ws + j;  // word j of the lane's row 0
        uint32_t yh[4], yl[4], yn[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            uint32_t h = 0, lo = 0, nn = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t w = *row;
                row += ws;
                const uint32_t xh = u >= 2 ? w << (u - 2) : w >> (2 - u);
                const uint32_t xl = u >= 1 ? w << (u - 1) : w >> 1;
                h |= xh & (0x01010101u << u);
                lo |= xl & (0x01010101u << u);
                if (WITH_N)
                    nn |= (n_bytes(w) >> 7) << u;
                else
                    seen |= w & keep;
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
    return seen;
}

// pack_transpose_by with the threads of the CTA in threadIdx.x order.
template <bool WITH_N, bool ALIGNED, int LANES = 8>
__device__ __forceinline__ uint32_t pack_transpose(const uint32_t *__restrict__ sm, int m, int rs,
                                                   size_t tile, int lane0,
                                                   uint32_t *__restrict__ packed,
                                                   uint32_t *__restrict__ nmask, int rot_step,
                                                   int nthreads)
{
    return pack_transpose_by<WITH_N, ALIGNED, LANES>(sm, m, rs, tile, lane0, packed, nmask,
                                                     rot_step, nthreads, (int)threadIdx.x);
}

// Per-lane rotation step c with c * (rs/4) = 32/lanes (mod 32) when such a c
// exists (then the lanes x 32/lanes position quads of a warp read 32
// distinct banks); 0 when the row stride rs is not a multiple of 4 or no
// such c exists.
__host__ __device__ inline int rotation_step(int rs, int lanes = 8)
{
    if (rs % 4)
        return 0;
    const int W = rs / 4, target = 32 / lanes;
    for (int c = 0; c < 32; ++c)
        if ((c * W) % 32 == target)
            return c;
    return 0;
}

// 16-byte global -> shared copies that run while the thread goes on
// (cp.async); a source size below 16 zero-fills the rest of the 16 bytes, and
// a size of 0 reads nothing.  wait<N> waits for this thread's copies of all
// but the N most recent groups.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, uint32_t src_bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One-dimensional bulk copies (cp.async.bulk, the TMA unit) that complete on
// an mbarrier in shared memory.  A bulk copy wants a 16-byte aligned source
// and destination and a size that is a multiple of 16 bytes.
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
// Makes initialised barriers visible to the copy engine.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// Orders this CTA's earlier shared-memory accesses before later bulk copies
// into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// Arrives once and announces `bytes` more to come from bulk copies; with
// bytes == 0 the arrival alone completes the phase.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *smem_dst, const void *gsrc, uint32_t bytes,
                                              uint64_t *bar)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
        ::"r"(d), "l"(gsrc), "r"(bytes), "r"(b) : "memory");
}
// One test of the phase; while it is incomplete the thread may sleep in the
// instruction, for at most about kSuspendNs (it wakes when the phase
// completes), so waiting warps take no issue slots from working ones.
constexpr uint32_t kSuspendNs = 100000;
// The same bulk copy with an L2 eviction policy (from createpolicy).
__device__ __forceinline__ void bulk_copy_g2s_hint(void *smem_dst, const void *gsrc,
                                                   uint32_t bytes, uint64_t *bar,
                                                   uint64_t policy)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1], %2, [%3], %4;\n"
        ::"r"(d), "l"(gsrc), "r"(bytes), "r"(b), "l"(policy) : "memory");
}
// L2 policy: lines brought in go first when L2 needs room (data read once).
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(a), "r"(parity), "n"(kSuspendNs) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// Tests a bounded wait makes at most: one test sleeps at most kSuspendNs,
// so the wait ends within about 2 s even should the timer stand still.
constexpr int kMaxWaitTests = 20000;
static_assert((uint64_t)kMaxWaitTests * kSuspendNs <= 2100000000ull,
              "a bounded wait must end within about 2 s");
// Waits for the phase of `bar` with the given parity to complete; gives up
// (false) after about a second by the global timer, or after kMaxWaitTests
// tests, whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = globaltimer_ns();
    for (int it = 0; it < kMaxWaitTests; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (globaltimer_ns() - t0 > 1000000000ull)
            return false;
    }
    return false;
}

}  // namespace packdev
}  // namespace shouji
