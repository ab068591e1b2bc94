// shouji_magnet: the MAGNET filter (Supplementary Sec. 7, Algorithms 3 and 4
// of the paper) on the packed pairs of shouji_pack.
//
// MAGNET looks for at most E+1 non-overlapping common subsequences of a
// pair.  It takes the longest run of zeros over all 2E+1 diagonals of the
// neighborhood map inside the current column range, writes it as zeros into
// the MAGNET bit-vector (all ones at the start), keeps the column just
// before and just after it out of the search (encapsulation: those edits
// stay visible), and solves the range right of the run and then the range
// left of it the same way.  The first run must reach ceil((m-E)/(E+1))
// columns, or the pair is rejected at once.  The pair is accepted iff the
// MAGNET vector holds at most E ones.
//
// GPU form.  The recursion follows each pair's own data, so one thread runs
// one pair, and the pair lives in registers as column masks (bit c % 32 of
// word c / 32 = column c):
//  - a warp reads the packed words of its 32 pairs 32 positions at a time
//    (lane i: position 32w + i) and turns them around with a 32 x 32 bit
//    transpose across the warp, so that lane b holds word w of pair b;
//  - diagonal d's matches are "P moved by d columns equals T" on both
//    bit-planes, with columns out of the band, N columns and columns outside
//    the range cleared: six logic ops per word;
//  - the longest run of ones of a mask comes from the ladder A_1 = x,
//    A_2L = A_L & (A_L >> L), which stops at its first empty level and so
//    bounds the run to [2^(k-1), 2^k); a diagonal whose bound cannot beat the
//    best run so far is dropped there, otherwise the descent
//    A_(L+h) = A_h & (A_L >> h) over the stored levels gives the exact
//    length, and the lowest set bit of A_L the leftmost start;
//  - the recursion is an explicit stack of column ranges: the left range is
//    pushed under the right one, so the right range and all of its own
//    subranges are solved first, as in Algorithm 4.
// Ties between runs of one length go, in this order, to upper_1, lower_1,
// upper_2, lower_2, ..., and last to the main diagonal; within a diagonal to
// the leftmost run.
#include "shouji_internal.cuh"

namespace shouji {
namespace {

constexpr int kMagnetThreads = 128;
constexpr int kMaxStack = SHOUJI_MAX_E + 3;  // 1 + one net push per extraction

__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t lowhalf = s == 16 ? 0x0000FFFFu
                                 : s == 8 ? 0x00FF00FFu
                                 : s == 4 ? 0x0F0F0F0Fu
                                 : s == 2 ? 0x33333333u
                                          : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, s);
        const bool up = (lane & s) != 0;
        const uint32_t keep = up ? ~lowhalf : lowhalf;
        const uint32_t t = up ? (y >> s) : (y << s);
        x = (x & keep) | (t & ~keep);
    }
    return x;
}

// Bits [lo, hi] of the column range, restricted to word w.
__device__ __forceinline__ uint32_t span_mask(int lo, int hi, int w)
{
    const int a = lo - 32 * w, b = hi - 32 * w;
    if (b < 0 || a > 31 || a > b)
        return 0u;
    const uint32_t upto = b >= 31 ? 0xFFFFFFFFu : ((2u << b) - 1u);
    return upto & (0xFFFFFFFFu << (a < 0 ? 0 : a));
}

template <int W>
__device__ __forceinline__ bool any(const uint32_t (&x)[W])
{
    uint32_t o = x[0];
#pragma unroll
    for (int w = 1; w < W; ++w)
        o |= x[w];
    return o != 0u;
}

// Number of ladder levels: A_1 ... A_(2^(LV-1)), enough for runs up to
// min(32 W, 255) columns.
template <int W>
__host__ __device__ constexpr int ladder_levels()
{
    return W == 1 ? 6 : W <= 3 ? 7 : 8;
}

// Word w of x moved h columns down (column c of the result = column c + h of
// x), zero fill; h is a power of two known after unrolling.
template <int W>
__device__ __forceinline__ uint32_t down_word(const uint32_t *x, int h, int w)
{
    if (h >= 32) {
        const int q = h / 32;
        return (w + q < W) ? x[w + q] : 0u;
    }
    return __funnelshift_r(x[w], w + 1 < W ? x[w + 1] : 0u, h);
}

// Exact run length from the ladder whose top non-empty level is K-1:
// A_(L+h) = A_h & (A_L >> h) for h = 2^(K-2) ... 1.
template <int W, int LV, int K>
__device__ __forceinline__ void descend(const uint32_t *lv, uint32_t (&cur)[W], int &L)
{
#pragma unroll
    for (int w = 0; w < W; ++w)
        cur[w] = lv[(K - 1) * W + w];
    L = 1 << (K - 1);
#pragma unroll
    for (int j = K - 2; j >= 0; --j) {
        uint32_t t[W], o = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            t[w] = lv[j * W + w] & down_word<W>(cur, 1 << j, w);
            o |= t[w];
        }
        if (o) {
#pragma unroll
            for (int w = 0; w < W; ++w)
                cur[w] = t[w];
            L += 1 << j;
        }
    }
}

// Longest run of ones in x and its leftmost start, if it beats `floor_len`
// (or ties with it when tie_ok); otherwise 0.  The descent is dispatched on
// the ladder height k so that every level is read at a constant index and
// the ladder stays in registers.
template <int W>
__device__ __forceinline__ int longest_run(const uint32_t (&x)[W], int floor_len, bool tie_ok,
                                           int &start)
{
    constexpr int LV = ladder_levels<W>();
    uint32_t lv[LV * W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        lv[w] = x[w];
    if (!any(x))
        return 0;
    int k = 1;  // levels 0 .. k-1 are non-empty
#pragma unroll
    for (int j = 1; j < LV; ++j) {
        if (k == j) {
            uint32_t o = 0u;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                lv[j * W + w] = lv[(j - 1) * W + w] & down_word<W>(lv + (j - 1) * W, 1 << (j - 1), w);
                o |= lv[j * W + w];
            }
            if (o)
                k = j + 1;
        }
    }
    const int bound = (1 << k) - 1;
    if (bound < floor_len || (bound == floor_len && !tie_ok))
        return 0;
    uint32_t cur[W];
    int L = 0;
    switch (k) {
#define SHOUJI_DESCENT_CASE(K)                                   \
    case K:                                                      \
        if (K <= LV)                                             \
            descend<W, LV, (K <= LV ? K : 1)>(lv, cur, L);       \
        break;
        SHOUJI_DESCENT_CASE(1)
        SHOUJI_DESCENT_CASE(2)
        SHOUJI_DESCENT_CASE(3)
        SHOUJI_DESCENT_CASE(4)
        SHOUJI_DESCENT_CASE(5)
        SHOUJI_DESCENT_CASE(6)
        SHOUJI_DESCENT_CASE(7)
        SHOUJI_DESCENT_CASE(8)
#undef SHOUJI_DESCENT_CASE
    }
    if (L < floor_len || (L == floor_len && !tie_ok))
        return 0;
    int s = 0;
#pragma unroll
    for (int w = W - 1; w >= 0; --w)
        if (cur[w])
            s = 32 * w + __ffs(cur[w]) - 1;
    start = s;
    return L;
}

template <int W, bool WITH_N>
__global__ void __launch_bounds__(kMagnetThreads)
magnet_kernel(const FilterArgs a, const int E)
{
    const int lane = threadIdx.x & 31;
    const size_t g = (size_t)blockIdx.x * (kMagnetThreads / 32) + (threadIdx.x >> 5);
    if (g >= groups_of(a.n_pairs))
        return;  // whole warp
    const int m = a.m;
    const size_t t = g / kLanes;
    const int l = (int)(g % kLanes);
    const size_t pair = g * 32 + lane;
    const bool live = pair < a.n_pairs;

    // The pair's sequences as column masks; Br = read columns that match
    // nothing (N, or past the end), Nt = reference N columns.
    uint32_t Rh[W], Rl[W], Th[W], Tl[W], Br[W], Nt[W], Mv[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int p = 32 * w + lane;
        uint2 r = make_uint2(0u, 0u), f = make_uint2(0u, 0u);
        uint32_t nr = 0u, nf = 0u;
        if (p < m) {
            const size_t idx = ((size_t)t * m + p) * kLanes + l;
            r = __ldg(a.reads + idx);
            f = __ldg(a.refs + idx);
            if (WITH_N) {
                nr = __ldg(a.reads_n + idx);
                nf = __ldg(a.refs_n + idx);
            }
        }
        Rh[w] = warp_transpose(r.x, lane);
        Rl[w] = warp_transpose(r.y, lane);
        Th[w] = warp_transpose(f.x, lane);
        Tl[w] = warp_transpose(f.y, lane);
        Mv[w] = span_mask(0, m - 1, w);
        Br[w] = ~Mv[w];
        Nt[w] = 0u;
        if (WITH_N) {
            Br[w] |= warp_transpose(nr, lane);
            Nt[w] = warp_transpose(nf, lane);
        }
    }

    int Ep = E;
    if (a.E_per_pair && live)
        Ep = min((int)__ldg(a.E_per_pair + pair), E);

    uint32_t V[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        V[w] = live ? Mv[w] : 0u;

    uint16_t stack[kMaxStack];
    int sp = 0;
    if (live)
        stack[sp++] = (uint16_t)((m - 1) << 8);  // range [0, m-1]
    int done = 0;                                // extractions so far
    const int first_min = m / (Ep + 1);          // ceil((m - E) / (E + 1))

    while (sp > 0 && done <= Ep) {
        const uint32_t range = stack[--sp];
        const int SI = (int)(range & 0xFFu), EI = (int)(range >> 8);
        uint32_t G[W];
#pragma unroll
        for (int w = 0; w < W; ++w)
            G[w] = span_mask(SI, EI, w) & ~Nt[w];

        uint32_t x[W];
        int s = 0;
        // Main diagonal: examined first for an early bound, ranked last.
#pragma unroll
        for (int w = 0; w < W; ++w)
            x[w] = ~((Rh[w] ^ Th[w]) | (Rl[w] ^ Tl[w]) | Br[w]) & G[w];
        int best_len = longest_run(x, 0, false, s);
        int best_s = s;
        bool best_main = best_len > 0;
        for (int j = 1; j <= Ep; ++j) {
            // upper_j: column c compares P[c - j] with T[c]
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint32_t h = __funnelshift_l(w ? Rh[w ? w - 1 : 0] : 0u, Rh[w], j);
                const uint32_t lo = __funnelshift_l(w ? Rl[w ? w - 1 : 0] : 0u, Rl[w], j);
                const uint32_t b = __funnelshift_l(w ? Br[w ? w - 1 : 0] : 0xFFFFFFFFu, Br[w], j);
                x[w] = ~((h ^ Th[w]) | (lo ^ Tl[w]) | b) & G[w];
            }
            int L = longest_run(x, best_len, best_main, s);
            if (L) {
                best_len = L;
                best_s = s;
                best_main = false;
            }
            // lower_j: column c compares P[c + j] with T[c]
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const int nx = w + 1 < W ? w + 1 : 0;
                const uint32_t h = __funnelshift_r(Rh[w], w + 1 < W ? Rh[nx] : 0u, j);
                const uint32_t lo = __funnelshift_r(Rl[w], w + 1 < W ? Rl[nx] : 0u, j);
                const uint32_t b = __funnelshift_r(Br[w], w + 1 < W ? Br[nx] : 0xFFFFFFFFu, j);
                x[w] = ~((h ^ Th[w]) | (lo ^ Tl[w]) | b) & G[w];
            }
            L = longest_run(x, best_len, best_main, s);
            if (L) {
                best_len = L;
                best_s = s;
                best_main = false;
            }
        }
        if (best_len == 0)
            continue;  // no zero in the range: nothing extracted
        if (done == 0 && best_len < first_min)
            break;     // early rejection; the vector is still all ones
        const int e = best_s + best_len - 1;
#pragma unroll
        for (int w = 0; w < W; ++w)
            V[w] &= ~span_mask(best_s, e, w);
        ++done;
        if (best_s - 2 >= SI)
            stack[sp++] = (uint16_t)(SI | ((best_s - 2) << 8));
        if (e + 2 <= EI)
            stack[sp++] = (uint16_t)((e + 2) | (EI << 8));
    }

    int ones = 0;
#pragma unroll
    for (int w = 0; w < W; ++w)
        ones += __popc(V[w]);
    const bool acc = live && ones <= Ep;
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, acc);
    if (lane == 0)
        a.accept[g] = bits;
    if (a.count && live)
        a.count[pair] = (uint8_t)ones;
    if (a.vectors) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t col = warp_transpose(V[w], lane);
            const int p = 32 * w + lane;
            if (p < m)
                a.vectors[((size_t)t * m + p) * kLanes + l] = col;
        }
    }
}

template <int W>
cudaError_t launch_W(const FilterArgs &a, int E, cudaStream_t s)
{
    const size_t groups = groups_of(a.n_pairs);
    const size_t warps_per_block = kMagnetThreads / 32;
    const unsigned blocks = (unsigned)((groups + warps_per_block - 1) / warps_per_block);
    if (a.reads_n)
        magnet_kernel<W, true><<<blocks, kMagnetThreads, 0, s>>>(a, E);
    else
        magnet_kernel<W, false><<<blocks, kMagnetThreads, 0, s>>>(a, E);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_magnet(const FilterArgs &a, int E, cudaStream_t s)
{
    switch ((a.m + 31) / 32) {
    case 1: return launch_W<1>(a, E, s);
    case 2: return launch_W<2>(a, E, s);
    case 3: return launch_W<3>(a, E, s);
    case 4: return launch_W<4>(a, E, s);
    case 5: return launch_W<5>(a, E, s);
    case 6: return launch_W<6>(a, E, s);
    case 7: return launch_W<7>(a, E, s);
    default: return launch_W<8>(a, E, s);
    }
}

}  // namespace shouji

using namespace shouji;

extern "C" shouji_status shouji_magnet(const uint32_t *reads, const uint32_t *refs,
                                       const uint32_t *reads_nmask, const uint32_t *refs_nmask,
                                       uint32_t m, size_t n_pairs, int E,
                                       const uint8_t *E_per_pair, uint32_t *out_accept,
                                       uint8_t *out_count, uint32_t *out_vectors, void *stream)
{
    if (m < 1 || m > SHOUJI_MAX_M || E < 0 || E > SHOUJI_MAX_E)
        return SHOUJI_EINVAL;
    if ((reads_nmask == nullptr) != (refs_nmask == nullptr))
        return SHOUJI_EINVAL;
    if (n_pairs == 0)
        return SHOUJI_OK;
    if (!reads || !refs || !out_accept)
        return SHOUJI_EINVAL;
    if ((uintptr_t)reads % 8 || (uintptr_t)refs % 8)
        return SHOUJI_EINVAL;
    FilterArgs a;
    a.reads = reinterpret_cast<const uint2 *>(reads);
    a.refs = reinterpret_cast<const uint2 *>(refs);
    a.reads_n = reads_nmask;
    a.refs_n = refs_nmask;
    a.E_per_pair = E_per_pair;
    a.accept = out_accept;
    a.count = out_count;
    a.vectors = out_vectors;
    a.n_pairs = n_pairs;
    a.m = (int)m;
    return cuda_status(launch_magnet(a, E, (cudaStream_t)stream));
}
