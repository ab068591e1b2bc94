// The Shouji filter kernel (arXiv 1809.07858, Sec. 2.2), bit-sliced across
// pairs: one thread filters 32 pairs at once.  Every 32-bit register holds
// one bit position of 32 pairs (bit b = pair b of the thread's group), so a
// single LOP3 advances all 32 pairs; no instruction depends on the data, and
// the per-pair serial chain of the paper's Step 2 becomes 32 pairs per step.
//
// Per window c (c = 0..m-1) and pair, the paper's work is:
//   Step 1 (neighborhood map, Eq. 1): diagonal d in [-E, E] has, at column p,
//     the mismatch bit M_d[p] = [P[p-d] != T[p]] (1 outside the band, 1 past
//     the end).  With the 2-bit codes, M = (Th ^ Ph) | (Tl ^ Pl) (| N masks).
//   Step 2a (search window, Sec. 2.2.2): the segment M_d[c..c+3] with the
//     most zeros, ties to the first with a leading zero, in the order lower_1,
//     upper_1, ..., lower_E, upper_E, then the main diagonal with strictly
//     more zeros.  Keys are compared without counting: with a = candidate,
//     b = current choice, "a wins" <=> 2(ones(b) - ones(a)) + 3(b0 - a0) > 0,
//     evaluated on the full-adder sum/carry of bits 1..3 of each segment.
//   Step 2b (Shouji bit-vector): S starts as all ones; window c writes Z into
//     S[c..c+3] iff Z has strictly more zeros.  Only windows >= c can write
//     S[c+3], so before window c the live state is (S[c], S[c+1], S[c+2]) and
//     S[c+3] = 1; after window c, S[c] is final.  The test "Z has more zeros"
//     is ones(Z) <= ones(S[c..c+2]), again from full-adder bits.
//   Step 3 (Sec. 2.2.3): the final S bits are summed in a bit-sliced 8-bit
//     counter; accept iff count <= E.
//
// Windows are processed in chunks of U; a chunk recomputes the U+3 map
// columns it needs for each diagonal from the packed words (loads go through
// the read-only cache; the footprint per warp is a few KB).
#pragma once

#include "shouji_internal.cuh"

namespace shouji {
namespace filt {

constexpr int kThreads = 128;
#ifndef SHOUJI_FILTER_U
#define SHOUJI_FILTER_U 4
#endif

__device__ __forceinline__ uint32_t maj3(uint32_t a, uint32_t b, uint32_t c)
{
    return (a & b) | (a & c) | (b & c);
}

// Current choice of one window: bits z0..z3 (1 = mismatch) and the full-adder
// sum/carry of z1..z3 (ones(z) = z0 + zs + 2*zc).
struct Pick {
    uint32_t z0, z1, z2, z3, zs, zc;
};

__device__ __forceinline__ Pick make_pick(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3)
{
    Pick p;
    p.z0 = a0;
    p.z1 = a1;
    p.z2 = a2;
    p.z3 = a3;
    p.zs = a1 ^ a2 ^ a3;
    p.zc = maj3(a1, a2, a3);
    return p;
}

// Offer candidate segment a (a0..a3) to the window's current choice b under the
// rule "more zeros wins; on a tie a leading zero beats a leading one".
// With u = ones(b1..b3) + zeros(a1..a3) in [0, 6] and v = b0 + (1 - a0):
// a wins <=> 2u + 3v >= 10, i.e. v=2: u>=2;  v=1: u>=4;  v=0: u>=5.
__device__ __forceinline__ void offer(Pick &b, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3)
{
    const uint32_t as = a1 ^ a2 ^ a3;
    const uint32_t ac = maj3(a1, a2, a3);
    // zeros(a1..a3) = ~as + 2 ~ac ; u = x0 + 2 (x1 + b.zc + ~ac) = x0 + 2 y0 + 4 y1
    const uint32_t x0 = b.zs ^ ~as;
    const uint32_t x1 = b.zs & ~as;
    const uint32_t y0 = x1 ^ b.zc ^ ~ac;
    const uint32_t y1 = maj3(x1, b.zc, ~ac);
    const uint32_t win = (y1 & (b.z0 | ~a0 | x0 | y0)) | (~y1 & b.z0 & ~a0 & y0);
    b.z0 = (win & a0) | (~win & b.z0);
    b.z1 = (win & a1) | (~win & b.z1);
    b.z2 = (win & a2) | (~win & b.z2);
    b.z3 = (win & a3) | (~win & b.z3);
    b.zs = (win & as) | (~win & b.zs);
    b.zc = (win & ac) | (~win & b.zc);
}

// The main diagonal replaces the choice only with strictly more zeros:
// ones(z) > ones(main) <=> ones(z) + ones(~main) >= 5, with
// ones(~main) = ~m0 + ~ms + 2 ~mc (ms, mc: full adder of main bits 1..3).
// Summing z0 + ~m0 + zs -> (f0, f1), f0 + ~ms -> (g0, g1), g1 + f1 + zc ->
// (k0, k1): total = g0 + 2 h with h = k0 + 2 k1 + ~mc, and total >= 5 <=>
// h >= 3 or (h >= 2 and g0).
__device__ __forceinline__ void offer_main(Pick &b, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3)
{
    const uint32_t ms = a1 ^ a2 ^ a3;
    const uint32_t mc = maj3(a1, a2, a3);
    const uint32_t f0 = b.z0 ^ ~a0 ^ b.zs;
    const uint32_t f1 = maj3(b.z0, ~a0, b.zs);
    const uint32_t g0 = f0 ^ ~ms;
    const uint32_t g1 = f0 & ~ms;
    const uint32_t k0 = g1 ^ f1 ^ b.zc;
    const uint32_t k1 = maj3(g1, f1, b.zc);
    const uint32_t gt = (k1 & (k0 | ~mc)) | (g0 & (k1 | (k0 & ~mc)));
    b.z0 = (gt & a0) | (~gt & b.z0);
    b.z1 = (gt & a1) | (~gt & b.z1);
    b.z2 = (gt & a2) | (~gt & b.z2);
    b.z3 = (gt & a3) | (~gt & b.z3);
    b.zs = (gt & ms) | (~gt & b.zs);
    b.zc = (gt & mc) | (~gt & b.zc);
}

// Bit-sliced 8-bit counter += x (3-bit value x2 x1 x0).
__device__ __forceinline__ void counter_add3(uint32_t (&C)[8], uint32_t x0, uint32_t x1, uint32_t x2)
{
    uint32_t k = C[0] & x0;
    C[0] ^= x0;
    uint32_t t = C[1] ^ x1;
    uint32_t k2 = maj3(C[1], x1, k);
    C[1] = t ^ k;
    k = k2;
    t = C[2] ^ x2;
    k2 = maj3(C[2], x2, k);
    C[2] = t ^ k;
    k = k2;
#pragma unroll
    for (int i = 3; i < 8; ++i) {
        const uint32_t c = C[i] & k;
        C[i] ^= k;
        k = c;
    }
}

// 4x4 byte transpose: out[q] byte u = in[u] byte q.
__device__ __forceinline__ void byte_transpose4(uint32_t y0, uint32_t y1, uint32_t y2, uint32_t y3,
                                                uint32_t out[4])
{
    const uint32_t a = __byte_perm(y0, y1, 0x5140);
    const uint32_t b = __byte_perm(y0, y1, 0x7362);
    const uint32_t c = __byte_perm(y2, y3, 0x5140);
    const uint32_t d = __byte_perm(y2, y3, 0x7362);
    out[0] = __byte_perm(a, c, 0x5410);
    out[1] = __byte_perm(a, c, 0x7632);
    out[2] = __byte_perm(b, d, 0x5410);
    out[3] = __byte_perm(b, d, 0x7632);
}

// Transpose of the 8x8 bit matrix held in a 64-bit word (bit 8r + c <->
// bit 8c + r), by three rounds of masked swaps (Hacker's Delight, 7-3).
__device__ __forceinline__ uint64_t bit_transpose8(uint64_t x)
{
    uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x = x ^ t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x = x ^ t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x = x ^ t ^ (t << 28);
    return x;
}

// Bit-sliced 8-bit counts (plane k, bit b = bit k of pair b's count) to one
// byte per pair: cw[q] byte u = count of pair 4q + u.
__device__ __forceinline__ void counts_to_bytes(const uint32_t (&C)[8], uint32_t (&cw)[8])
{
    uint32_t lo[4], hi[4];
    byte_transpose4(C[0], C[1], C[2], C[3], lo);  // lo[j] byte k = byte j of C[k]
    byte_transpose4(C[4], C[5], C[6], C[7], hi);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        // bit 8k + i = bit k of the count of pair 8j + i
        const uint64_t x = bit_transpose8(((uint64_t)hi[j] << 32) | lo[j]);
        cw[2 * j] = (uint32_t)x;
        cw[2 * j + 1] = (uint32_t)(x >> 32);
    }
}

// Accept bits for a constant threshold: bit b = (count of pair b) <= E.
template <int E>
__device__ __forceinline__ uint32_t le_const(const uint32_t (&C)[8])
{
    uint32_t gt = 0u, eq = ~0u;
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        if ((E >> k) & 1) {
            eq &= C[k];
        } else {
            gt |= eq & C[k];
            eq &= ~C[k];
        }
    }
    return ~gt;
}

// Per-thread view of the packed data of one group of 32 pairs.
struct View {
    const uint2 *rd, *rf;       // position p at [p * 32]
    const uint32_t *rdn, *rfn;  // N masks (may be null)
    uint32_t *vec;              // Shouji vectors out (may be null), [c * 32]
    int m;
};

// Loads of packed words: through the read-only cache, or (COHERENT) as plain
// loads, for words that another warp of the same CTA wrote earlier in the
// same kernel.
template <bool COHERENT, class T>
__device__ __forceinline__ T ldp(const T *p)
{
    if constexpr (COHERENT)
        return *p;
    else
        return __ldg(p);
}

// Map columns that a chunk hands to the next one: window c needs columns
// c..c+3, so consecutive chunks of U windows share 3 columns per diagonal.
// Keeping them in registers saves 3 of every U+3 map evaluations; for large
// E the 3(2E+1) extra live registers cost more than they save, and the
// shared columns are recomputed instead.
#ifndef SHOUJI_CARRY_MAX_E
#define SHOUJI_CARRY_MAX_E 15
#endif
#ifndef SHOUJI_LARGE_E_MIN_BLOCKS
#define SHOUJI_LARGE_E_MIN_BLOCKS 1
#endif

template <int E>
struct Carry {
    static constexpr bool kOn = E <= SHOUJI_CARRY_MAX_E;
    uint32_t M[kOn ? 2 * E + 1 : 1][3];
};

// One chunk of U windows starting at c0.
//   BOUNDS: columns and read positions may fall outside [0, m) (edge chunks);
//           an unbounded chunk needs every column it evaluates and every read
//           position those columns touch inside [0, m).
//   MASKS:  0 none; 1 N masks (of reads and refs); 2 N masks that may be
//           absent and per-pair thresholds.
// With a carry, the chunk evaluates the U columns c0+3..c0+U+2 and takes
// c0..c0+2 from the carry; without, it evaluates all U+3 columns c0..c0+U+2.
template <int E, int U, bool BOUNDS, int MASKS, bool COHERENT = false>
__device__ __forceinline__ void chunk(const View &v, const uint32_t (&inactive)[E + 1], int c0,
                                      Carry<E> &carry, uint32_t &s0, uint32_t &s1, uint32_t &s2,
                                      uint32_t (&C)[8])
{
    constexpr bool CARRY = Carry<E>::kOn;
    constexpr int K0 = CARRY ? 3 : 0;   // first evaluated column offset
    constexpr int NC = U + 3 - K0;      // evaluated columns c0+K0 .. c0+U+2
    constexpr int NR = NC + 2 * E;      // read positions c0+K0-E .. c0+U+2+E
    uint32_t th[NC], tl[NC], tx[MASKS ? NC : 1];
    uint32_t rh[NR], rl[NR], rx[MASKS ? NR : 1];
    // level 1 always has both N masks; level 2 may have none
    const bool nm = MASKS == 1 || (MASKS == 2 && v.rfn != nullptr);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int p = c0 + K0 + k;
        const bool ok = !BOUNDS || p < v.m;
        const uint2 w = ok ? ldp<COHERENT>(v.rf + (size_t)p * 32) : make_uint2(0u, 0u);
        th[k] = w.x;
        tl[k] = w.y;
        if constexpr (MASKS != 0)
            tx[k] = (ok && nm) ? ldp<COHERENT>(v.rfn + (size_t)p * 32) : 0u;
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int q = c0 + K0 - E + i;
        const bool ok = !BOUNDS || (q >= 0 && q < v.m);
        const uint2 w = ok ? ldp<COHERENT>(v.rd + (size_t)q * 32) : make_uint2(0u, 0u);
        rh[i] = w.x;
        rl[i] = w.y;
        if constexpr (MASKS != 0)
            rx[i] = (ok && nm) ? ldp<COHERENT>(v.rdn + (size_t)q * 32) : 0u;
    }

    // Mismatch bits of diagonal d at evaluated column k (column c0+K0+k).
    auto column = [&](int d, int k) -> uint32_t {
        const int i = k - d + E;
        uint32_t x = (th[k] ^ rh[i]) | (tl[k] ^ rl[i]);
        if constexpr (MASKS != 0)
            x |= tx[k] | rx[i];
        if constexpr (MASKS == 2)
            x |= inactive[d < 0 ? -d : d];
        if constexpr (BOUNDS) {
            const int p = c0 + K0 + k, q = p - d;
            if (p >= v.m || q < 0 || q >= v.m)
                x = ~0u;
        }
        return x;
    };
    // All U+3 columns of diagonal d for this chunk; the last 3 become the
    // next chunk's carry.
    auto columns = [&](int d, uint32_t (&M)[U + 3]) {
        if constexpr (CARRY) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                M[k] = carry.M[d + E][k];
        }
#pragma unroll
        for (int k = 0; k < NC; ++k)
            M[K0 + k] = column(d, k);
        if constexpr (CARRY) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                carry.M[d + E][k] = M[U + k];
        }
    };

    Pick pick[U];
    if constexpr (E == 0) {
        uint32_t M[U + 3];
        columns(0, M);
#pragma unroll
        for (int w = 0; w < U; ++w)
            pick[w] = make_pick(M[w], M[w + 1], M[w + 2], M[w + 3]);
    } else {
        {
            uint32_t M[U + 3];
            columns(-1, M);
#pragma unroll
            for (int w = 0; w < U; ++w)
                pick[w] = make_pick(M[w], M[w + 1], M[w + 2], M[w + 3]);
        }
#pragma unroll
        for (int j = 1; j <= E; ++j) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int d = side ? j : -j;
                if (d == -1)
                    continue;
                uint32_t M[U + 3];
                columns(d, M);
#pragma unroll
                for (int w = 0; w < U; ++w)
                    offer(pick[w], M[w], M[w + 1], M[w + 2], M[w + 3]);
            }
        }
        uint32_t M[U + 3];
        columns(0, M);
#pragma unroll
        for (int w = 0; w < U; ++w)
            offer_main(pick[w], M[w], M[w + 1], M[w + 2], M[w + 3]);
    }

    // Step 2b: the Shouji bit-vector, window by window.
    uint32_t out[U];
#pragma unroll
    for (int w = 0; w < U; ++w) {
        const Pick &z = pick[w];
        if (c0 + w < v.m) {
            const uint32_t ns = ~(s0 ^ s1 ^ s2);    // parity of zeros(s0..s2)
            const uint32_t nc = ~maj3(s0, s1, s2);  // carry of zeros(s0..s2)
            const uint32_t w1 = maj3(z.z0, z.zs, ns);
            const uint32_t upd = ~maj3(w1, z.zc, nc);  // ones(Z) <= ones(s0..s2)
            out[w] = (upd & z.z0) | (~upd & s0);
            s0 = (upd & z.z1) | (~upd & s1);
            s1 = (upd & z.z2) | (~upd & s2);
            s2 = z.z3 | ~upd;
            if (v.vec)
                v.vec[(size_t)(c0 + w) * 32] = out[w];
        } else {
            out[w] = 0u;
        }
    }
    // Step 3: add the U final bits to the counter (U = 4: one 3-bit sum).
#pragma unroll
    for (int w = 0; w < U; w += 4) {
        const uint32_t fs = out[w] ^ out[w + 1] ^ out[w + 2];
        const uint32_t fc = maj3(out[w], out[w + 1], out[w + 2]);
        const uint32_t x0 = fs ^ out[w + 3];
        const uint32_t t = fs & out[w + 3];
        counter_add3(C, x0, fc ^ t, fc & t);
    }
}

// Columns 0..2 of every diagonal: the carry the first chunk starts from.
template <int E, int MASKS, bool COHERENT = false>
__device__ __forceinline__ void carry_prologue(const View &v, const uint32_t (&inactive)[E + 1],
                                               Carry<E> &carry)
{
    if constexpr (Carry<E>::kOn) {
#pragma unroll
        for (int d = -E; d <= E; ++d) {
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const int q = p - d;
                uint32_t x = ~0u;
                if (p < v.m && q >= 0 && q < v.m) {
                    const uint2 t = ldp<COHERENT>(v.rf + (size_t)p * 32);
                    const uint2 r = ldp<COHERENT>(v.rd + (size_t)q * 32);
                    x = (t.x ^ r.x) | (t.y ^ r.y);
                    if constexpr (MASKS != 0) {
                        if (v.rfn)
                            x |= ldp<COHERENT>(v.rfn + (size_t)p * 32) |
                                 ldp<COHERENT>(v.rdn + (size_t)q * 32);
                    }
                    if constexpr (MASKS == 2)
                        x |= inactive[d < 0 ? -d : d];
                }
                carry.M[d + E][p] = x;
            }
        }
    }
}

// The whole filter for one group of 32 pairs: every window of the group's
// m columns; C receives the bit-sliced 8-bit counts of ones.
template <int E, int U, int MASKS, bool COHERENT = false>
__device__ __forceinline__ void filter_group(const View &v, const uint32_t (&inactive)[E + 1],
                                             uint32_t (&C)[8])
{
    static_assert(U % 4 == 0, "U must be a multiple of 4");
    uint32_t s0 = ~0u, s1 = ~0u, s2 = ~0u;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        C[i] = 0u;
    const int m = v.m;
    Carry<E> carry;
    carry_prologue<E, MASKS, COHERENT>(v, inactive, carry);
    constexpr int K0 = Carry<E>::kOn ? 3 : 0;
    for (int c0 = 0; c0 < m; c0 += U) {
        if ((c0 + K0 - E >= 0) && (c0 + U + 2 + E < m))
            chunk<E, U, false, MASKS, COHERENT>(v, inactive, c0, carry, s0, s1, s2, C);
        else
            chunk<E, U, true, MASKS, COHERENT>(v, inactive, c0, carry, s0, s1, s2, C);
    }
}

// Minimum resident CTAs per SM requested from ptxas (caps registers) for
// thresholds above 8.
template <int E>
constexpr int min_blocks() { return E > 8 ? SHOUJI_LARGE_E_MIN_BLOCKS : 1; }

template <int E, int U, int MASKS>
__global__ void __launch_bounds__(kThreads, min_blocks<E>())
filter_kernel(FilterArgs a)
{
    const size_t g = (size_t)blockIdx.x * kThreads + threadIdx.x;  // group of 32 pairs
    const size_t n_groups = groups_of(a.n_pairs);
    if (g >= n_groups)
        return;
    const size_t tile = g / kLanes;
    const int lane = (int)(g % kLanes);
    const int m = a.m;
    const size_t base = tile * (size_t)m * kLanes + lane;
    const size_t first = g * 32;
    const size_t left = a.n_pairs - first;

    View v;
    v.rd = a.reads + base;
    v.rf = a.refs + base;
    v.rdn = a.reads_n ? a.reads_n + base : nullptr;
    v.rfn = a.refs_n ? a.refs_n + base : nullptr;
    v.vec = a.vectors ? a.vectors + base : nullptr;
    v.m = m;

    // Per-pair thresholds: inactive[j] bit b = pair b's threshold is below j,
    // so diagonals +-j are all mismatches for it (they can then never win).
    uint32_t inactive[E + 1];
#pragma unroll
    for (int j = 0; j <= E; ++j)
        inactive[j] = 0u;
    if (MASKS == 2 && a.E_per_pair) {
        for (int b = 0; b < 32 && (size_t)b < left; ++b) {
            const int e = a.E_per_pair[first + b];
#pragma unroll
            for (int j = 1; j <= E; ++j)
                inactive[j] |= (uint32_t)(e < j) << b;
        }
    }

    uint32_t C[8];
    filter_group<E, U, MASKS>(v, inactive, C);

    // Per-pair counts and the accept word.
    uint32_t cw[8];
    counts_to_bytes(C, cw);
    uint32_t acc = le_const<E>(C);
    if (MASKS == 2 && a.E_per_pair) {
        acc = 0u;
        for (int b = 0; b < 32 && (size_t)b < left; ++b) {
            const uint32_t cnt = (cw[b >> 2] >> (8 * (b & 3))) & 0xFFu;
            const uint32_t e = a.E_per_pair[first + b];
            acc |= (uint32_t)(cnt <= e && cnt <= (uint32_t)E) << b;
        }
    }
    if (left < 32)
        acc &= (1u << left) - 1u;
    a.accept[g] = acc;
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
}

template <int E>
cudaError_t launch_E(const FilterArgs &a, cudaStream_t s)
{
    constexpr int U = SHOUJI_FILTER_U;
    const size_t groups = groups_of(a.n_pairs);
    const size_t blocks = (groups + kThreads - 1) / kThreads;
    if (a.E_per_pair)
        filter_kernel<E, U, 2><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    else if (a.reads_n)
        filter_kernel<E, U, 1><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    else
        filter_kernel<E, U, 0><<<(unsigned)blocks, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace filt

template <int E>
cudaError_t launch_filter_E(const FilterArgs &a, cudaStream_t s)
{
    return filt::launch_E<E>(a, s);
}

}  // namespace shouji
