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
//  - runs are measured with the ladder A_1 = x, A_2L = A_L & (A_L >> L): the
//    first empty level bounds the longest run to [2^(k-1), 2^k), the descent
//    A_(L+h) = A_h & (A_L >> h) gives its exact length, and the lowest set
//    bit of A_L its leftmost start;
//  - lanes of a warp run different pairs, so the work is arranged to keep
//    them on the same instructions.  Every diagonal gets the same cheap test
//    (A_1 ... A_8), which settles runs shorter than 8 columns.  The few
//    diagonals with a longer run (about one to three per similar pair) are
//    walked by each lane from its own list: the first extraction records all
//    of their runs of 8 or more columns (the runs of A_8), and a later
//    extraction only clips that list to its range, running the cheap test
//    again only when no listed run of 8 reaches into the range.  A pair with
//    more long runs than the list holds uses the full ladder instead;
//  - the recursion is an explicit stack of column ranges: the left range is
//    pushed under the right one, so the right range and all of its own
//    subranges are solved first, as in Algorithm 4.
// Ties between runs of one length go, in this order, to upper_1, lower_1,
// upper_2, lower_2, ..., and last to the main diagonal; within a diagonal to
// the leftmost run.
#include "shouji_internal.cuh"

namespace shouji {
namespace {

// Two warps per CTA: a CTA holds its registers until its slowest warp is
// done, and smaller CTAs let an SM take new groups sooner.
constexpr int kMagnetThreads = 64;
constexpr int kMaxStack = SHOUJI_MAX_E + 3;  // 1 + one net push per extraction
constexpr int kMainRank = 2 * SHOUJI_MAX_E;  // after every upper_j and lower_j
constexpr int kLong = 8;                     // runs this long are listed
constexpr int kMaxRuns = 32;                 // listed runs per pair

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

// A run of length L on a diagonal of rank `rank` replaces the best run so far
// iff it is longer, or as long and of a lower rank.
__device__ __forceinline__ bool beats(int L, int rank, int best_len, int best_rank)
{
    return L > best_len || (L == best_len && rank < best_rank);
}

// The same with the leftmost-run rule inside one diagonal: of two equally
// long runs of the same diagonal the one that starts first is kept.
__device__ __forceinline__ bool beats_at(int L, int rank, int start, int best_len,
                                         int best_rank, int best_s)
{
    return L > best_len ||
           (L == best_len && (rank < best_rank || (rank == best_rank && start < best_s)));
}

// Longest run of ones in x and its leftmost start, or 0 when it cannot beat
// the best run so far.  `k` receives the ladder height (the run lies in
// [2^(k-1), 2^k), k = 0 for an empty x).  Every lane takes the same code
// path whatever its ladder height: levels a lane does not need are skipped
// by a predicate, not by a branch to other code.
template <int W>
__device__ __forceinline__ int longest_run(const uint32_t (&x)[W], int rank, int best_len,
                                           int best_rank, int &start, int &k)
{
    constexpr int LV = ladder_levels<W>();
    uint32_t lv[LV][W], top[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        lv[0][w] = top[w] = x[w];
    k = any(x) ? 1 : 0;
    if (k == 0)
        return 0;
#pragma unroll
    for (int j = 1; j < LV; ++j) {
        if (k == j) {  // A_(2^j) = A_(2^(j-1)) & (A_(2^(j-1)) >> 2^(j-1))
            uint32_t o = 0u;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                lv[j][w] = lv[j - 1][w] & down_word<W>(lv[j - 1], 1 << (j - 1), w);
                o |= lv[j][w];
            }
            if (o) {
                k = j + 1;
#pragma unroll
                for (int w = 0; w < W; ++w)
                    top[w] = lv[j][w];
            }
        }
    }
    if (!beats((1 << k) - 1, rank, best_len, best_rank))
        return 0;
    // Descent: A_(L+h) = A_h & (A_L >> h), h = 2^(k-2) ... 1.
    int L = 1 << (k - 1);
#pragma unroll
    for (int j = LV - 2; j >= 0; --j) {
        if (j < k - 1) {
            uint32_t t[W], o = 0u;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                t[w] = lv[j][w] & down_word<W>(top, 1 << j, w);
                o |= t[w];
            }
            if (o) {
#pragma unroll
                for (int w = 0; w < W; ++w)
                    top[w] = t[w];
                L += 1 << j;
            }
        }
    }
    if (!beats(L, rank, best_len, best_rank))
        return 0;
    int s = 0;
#pragma unroll
    for (int w = W - 1; w >= 0; --w)
        if (top[w])
            s = 32 * w + __ffs(top[w]) - 1;
    start = s;
    return L;
}

// One pair in flight: its sequences as column masks, its MAGNET vector and
// its recursion state.  Br = read columns that match nothing (N, or past the
// end of the read), Nt = reference N columns.
template <int W>
struct PairState {
    uint32_t Rh[W], Rl[W], Th[W], Tl[W], Br[W], Nt[W], V[W];
    uint64_t cand;  // diagonals with a run of at least kLong columns (bit = slot)
    int nruns;      // runs in PairStack::runs; -1 once they did not fit
    int Ep;         // the pair's threshold
    int done;       // extractions so far
    int sp;         // ranges on the stack
    bool rejected;  // the first run was too short
};

// The dynamically indexed part of a pair's state, kept apart from PairState
// so that the column masks stay in registers.  Diagonals are numbered by
// slot: 0 = main, 2j-1 = upper_j, 2j = lower_j.
struct PairStack {
    uint16_t range[kMaxStack];          // column ranges [lo | hi << 8]
    uint8_t len[2 * SHOUJI_MAX_E + 1];  // longest run of each diagonal over all columns
    uint32_t runs[kMaxRuns];            // runs of kLong or more: start | end << 8 | slot << 16
};

// Column masks of pair `lane` of group g (32 pairs of one tile lane), read
// 32 positions at a time and turned around by the warp transpose.  Every
// lane of the warp must take part.
template <int W, bool WITH_N>
__device__ __forceinline__ void load_group(const FilterArgs &a, size_t g, int lane,
                                           uint32_t (&P)[6][W])
{
    const int m = a.m;
    const size_t t = g / kLanes;
    const int l = (int)(g % kLanes);
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
        P[0][w] = warp_transpose(r.x, lane);
        P[1][w] = warp_transpose(r.y, lane);
        P[2][w] = warp_transpose(f.x, lane);
        P[3][w] = warp_transpose(f.y, lane);
        P[4][w] = WITH_N ? warp_transpose(nr, lane) : 0u;
        P[5][w] = WITH_N ? warp_transpose(nf, lane) : 0u;
    }
}

template <int W>
__device__ __forceinline__ void init_pair(PairState<W> &st, PairStack &sk,
                                          const uint32_t (&P)[6][W], int m, int Ep)
{
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const uint32_t mv = span_mask(0, m - 1, w);
        st.Rh[w] = P[0][w];
        st.Rl[w] = P[1][w];
        st.Th[w] = P[2][w];
        st.Tl[w] = P[3][w];
        st.Br[w] = P[4][w] | ~mv;
        st.Nt[w] = P[5][w];
        st.V[w] = mv;
    }
    st.cand = 0ull;
    st.nruns = 0;
    st.Ep = Ep;
    st.done = 0;
    st.rejected = false;
    sk.range[0] = (uint16_t)((m - 1) << 8);  // range [0, m-1]
    st.sp = 1;
}

// Rank of a slot in the order of preference between equally long runs:
// upper_j has rank 2(j-1), lower_j rank 2(j-1)+1, the main diagonal last.
__device__ __forceinline__ int rank_of(int slot) { return slot ? slot - 1 : kMainRank; }

// Matches of the diagonal in `slot` inside the columns of G.  The direction
// is a run-time value: the read is moved by a funnel shift whose operand
// pair and amount are chosen per lane (upper_j: up by j; lower_j: down by j;
// main: not moved).
template <int W>
__device__ __forceinline__ void build_any(const PairState<W> &st, const uint32_t (&G)[W],
                                          int slot, uint32_t (&x)[W])
{
    const int j = (slot + 1) >> 1;
    const bool up = (slot & 1) != 0;
    const int n = up ? 32 - j : j;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        const int pv = w ? w - 1 : 0, nx = w + 1 < W ? w + 1 : 0;
        const uint32_t hl = up ? (w ? st.Rh[pv] : 0u) : st.Rh[w];
        const uint32_t hh = up ? st.Rh[w] : (w + 1 < W ? st.Rh[nx] : 0u);
        const uint32_t ll = up ? (w ? st.Rl[pv] : 0u) : st.Rl[w];
        const uint32_t lh = up ? st.Rl[w] : (w + 1 < W ? st.Rl[nx] : 0u);
        const uint32_t bl = up ? (w ? st.Br[pv] : 0xFFFFFFFFu) : st.Br[w];
        const uint32_t bh = up ? st.Br[w] : (w + 1 < W ? st.Br[nx] : 0xFFFFFFFFu);
        const uint32_t h = __funnelshift_rc(hl, hh, n);
        const uint32_t lo = __funnelshift_rc(ll, lh, n);
        const uint32_t b = __funnelshift_rc(bl, bh, n);
        x[w] = ~((h ^ st.Th[w]) | (lo ^ st.Tl[w]) | b) & G[w];
    }
}

// The same with the direction fixed at compile time (0: main, 1: upper_j,
// -1: lower_j), for loops in which every lane examines the same diagonal.
template <int W, int DIR>
__device__ __forceinline__ void build_fixed(const PairState<W> &st, const uint32_t (&G)[W],
                                            int j, uint32_t (&x)[W])
{
#pragma unroll
    for (int w = 0; w < W; ++w) {
        uint32_t h, lo, b;
        if (DIR > 0) {         // column c compares P[c - j] with T[c]
            const int pv = w ? w - 1 : 0;
            h = __funnelshift_l(w ? st.Rh[pv] : 0u, st.Rh[w], j);
            lo = __funnelshift_l(w ? st.Rl[pv] : 0u, st.Rl[w], j);
            b = __funnelshift_l(w ? st.Br[pv] : 0xFFFFFFFFu, st.Br[w], j);
        } else if (DIR < 0) {  // column c compares P[c + j] with T[c]
            const int nx = w + 1 < W ? w + 1 : 0;
            h = __funnelshift_r(st.Rh[w], w + 1 < W ? st.Rh[nx] : 0u, j);
            lo = __funnelshift_r(st.Rl[w], w + 1 < W ? st.Rl[nx] : 0u, j);
            b = __funnelshift_r(st.Br[w], w + 1 < W ? st.Br[nx] : 0xFFFFFFFFu, j);
        } else {
            h = st.Rh[w];
            lo = st.Rl[w];
            b = st.Br[w];
        }
        x[w] = ~((h ^ st.Th[w]) | (lo ^ st.Tl[w]) | b) & G[w];
    }
}

// Longest run of ones in x if it is shorter than kLong columns: its exact
// length and leftmost start from the first levels of the ladder only
// (A_1, A_2, A_4, A_8).  Returns -1 when x has a run of kLong or more.
template <int W>
__device__ __forceinline__ int short_run(const uint32_t (&x)[W], int &start)
{
    uint32_t a1[W], a2[W], a4[W], a8[W];
    uint32_t o1 = 0u, o2 = 0u, o4 = 0u, o8 = 0u;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        a1[w] = x[w];
        o1 |= a1[w];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        a2[w] = a1[w] & down_word<W>(a1, 1, w);
        o2 |= a2[w];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        a4[w] = a2[w] & down_word<W>(a2, 2, w);
        o4 |= a4[w];
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
        a8[w] = a4[w] & down_word<W>(a4, 4, w);
        o8 |= a8[w];
    }
    if (o8)
        return -1;
    if (!o1)
        return 0;
    // top non-empty level and its length
    uint32_t cur[W];
    int L;
#pragma unroll
    for (int w = 0; w < W; ++w)
        cur[w] = o4 ? a4[w] : o2 ? a2[w] : a1[w];
    L = o4 ? 4 : o2 ? 2 : 1;
    // descent: + 2 (only from A_4), + 1 (from A_4 or A_2)
    if (o4) {
        uint32_t t[W], o = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            t[w] = a2[w] & down_word<W>(cur, 2, w);
            o |= t[w];
        }
        if (o) {
#pragma unroll
            for (int w = 0; w < W; ++w)
                cur[w] = t[w];
            L += 2;
        }
    }
    if (o2) {
        uint32_t t[W], o = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            t[w] = a1[w] & down_word<W>(cur, 1, w);
            o |= t[w];
        }
        if (o) {
#pragma unroll
            for (int w = 0; w < W; ++w)
                cur[w] = t[w];
            L += 1;
        }
    }
    int s = 0;
#pragma unroll
    for (int w = W - 1; w >= 0; --w)
        if (cur[w])
            s = 32 * w + __ffs(cur[w]) - 1;
    start = s;
    return L;
}

// The test of one diagonal for a run of kLong columns, in the first
// extraction and in every later one alike (one code path for all lanes,
// whatever step their pair is at).  A shorter run is settled here; a long
// one, which only the first extraction can meet, marks the diagonal as a
// candidate for the run list.  In later extractions this pass runs only when
// the listed runs leave the best run shorter than kLong: a diagonal is
// skipped when its bound (its longest short run over all columns, kLong - 1
// for a candidate, and never more than the range) cannot beat the best so
// far.  Candidates of a pair whose runs did not fit the list are left to the
// ladder.
template <int W, int DIR>
__device__ __forceinline__ void short_pass(PairState<W> &st, PairStack &sk,
                                           const uint32_t (&G)[W], int j, bool first,
                                           int range_len, int &best_len, int &best_s,
                                           int &best_rank)
{
    const int slot = DIR > 0 ? 2 * j - 1 : DIR < 0 ? 2 * j : 0;
    const int rank = rank_of(slot);
    const bool cand = ((st.cand >> slot) & 1ull) != 0;
    if (cand && (first || st.nruns < 0))
        return;
    if (!first) {
        const int ub = min(cand ? kLong - 1 : (int)sk.len[slot], range_len);
        if (ub < best_len || (ub == best_len && rank > best_rank))
            return;
    }
    uint32_t x[W];
    build_fixed<W, DIR>(st, G, j, x);
    int s = 0;
    const int L = short_run(x, s);
    if (L < 0) {
        if (first)
            st.cand |= 1ull << slot;
        return;
    }
    if (first)
        sk.len[slot] = (uint8_t)L;
    if (L > 0 && beats_at(L, rank, s, best_len, best_rank, best_s)) {
        best_len = L;
        best_s = s;
        best_rank = rank;
    }
}

// Word idx of a column mask, picked at a run-time index without indexing
// the register array (fill outside [0, W)).
template <int W>
__device__ __forceinline__ uint32_t word_at(const uint32_t (&P)[W], int idx, uint32_t fill)
{
    uint32_t v = fill;
#pragma unroll
    for (int w = 0; w < W; ++w)
        v = (w == idx) ? P[w] : v;
    return v;
}

// The columns of a later range that lies inside two words (ws, ws+1): the
// reference words there, the read words one word further on each side (a
// diagonal moves the read by up to 31 columns), and the range mask.
struct Window {
    uint32_t Rh[4], Rl[4], Br[4];  // read words ws-1 .. ws+2
    uint32_t Th[2], Tl[2], G[2];   // reference words ws, ws+1; range and N mask
    int base;                      // first column of word ws
};

template <int W>
__device__ __forceinline__ void make_window(const PairState<W> &st, int SI, int EI, Window &win)
{
    const int ws = SI >> 5;
    win.base = 32 * ws;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        win.Rh[k] = word_at(st.Rh, ws - 1 + k, 0u);
        win.Rl[k] = word_at(st.Rl, ws - 1 + k, 0u);
        win.Br[k] = word_at(st.Br, ws - 1 + k, 0xFFFFFFFFu);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        win.Th[k] = word_at(st.Th, ws + k, 0u);
        win.Tl[k] = word_at(st.Tl, ws + k, 0u);
        win.G[k] = span_mask(SI - win.base, EI - win.base, k) & ~word_at(st.Nt, ws + k, 0u);
    }
}

// short_pass for a later range inside a window: the same test on two words.
template <int DIR>
__device__ __forceinline__ void window_pass(const Window &win, uint64_t cand, const PairStack &sk,
                                            int j, int range_len, int &best_len, int &best_s,
                                            int &best_rank)
{
    const int slot = DIR > 0 ? 2 * j - 1 : DIR < 0 ? 2 * j : 0;
    const int rank = rank_of(slot);
    const bool is_cand = ((cand >> slot) & 1ull) != 0;
    const int ub = min(is_cand ? kLong - 1 : (int)sk.len[slot], range_len);
    if (ub < best_len || (ub == best_len && rank > best_rank))
        return;
    uint32_t x[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint32_t h, lo, b;
        if (DIR > 0) {  // read words ws+k-1, ws+k moved up by j
            h = __funnelshift_l(win.Rh[k], win.Rh[k + 1], j);
            lo = __funnelshift_l(win.Rl[k], win.Rl[k + 1], j);
            b = __funnelshift_l(win.Br[k], win.Br[k + 1], j);
        } else if (DIR < 0) {  // read words ws+k, ws+k+1 moved down by j
            h = __funnelshift_r(win.Rh[k + 1], win.Rh[k + 2], j);
            lo = __funnelshift_r(win.Rl[k + 1], win.Rl[k + 2], j);
            b = __funnelshift_r(win.Br[k + 1], win.Br[k + 2], j);
        } else {
            h = win.Rh[k + 1];
            lo = win.Rl[k + 1];
            b = win.Br[k + 1];
        }
        x[k] = ~((h ^ win.Th[k]) | (lo ^ win.Tl[k]) | b) & win.G[k];
    }
    int s = 0;
    const int L = short_run(x, s);
    if (L <= 0)
        return;  // no zero, or (impossible here) a run of kLong
    s += win.base;
    if (beats_at(L, rank, s, best_len, best_rank, best_s)) {
        best_len = L;
        best_s = s;
        best_rank = rank;
    }
}

// Lowest set bit of a column mask (32 W when empty).
template <int W>
__device__ __forceinline__ int lowest(const uint32_t (&y)[W])
{
    int p = 32 * W;
#pragma unroll
    for (int w = W - 1; w >= 0; --w)
        if (y[w])
            p = 32 * w + __ffs(y[w]) - 1;
    return p;
}

// First extraction, one candidate diagonal: its runs of kLong columns or more
// are the runs of A_8 = x & (x >> 1) & ... & (x >> 7), each lengthened by
// kLong - 1 columns.  They are walked from the left, appended to the run list
// and offered as the best run.  Returns the longest.  When the list is full
// the pair turns to the ladder for every candidate (nruns = -1).
template <int W>
__device__ __forceinline__ int list_runs(PairState<W> &st, PairStack &sk,
                                         const uint32_t (&x)[W], int slot, int &best_len,
                                         int &best_s, int &best_rank)
{
    uint32_t y[W], t[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        t[w] = x[w] & down_word<W>(x, 1, w);
#pragma unroll
    for (int w = 0; w < W; ++w)
        y[w] = t[w] & down_word<W>(t, 2, w);
#pragma unroll
    for (int w = 0; w < W; ++w)
        t[w] = y[w] & down_word<W>(y, 4, w);
#pragma unroll
    for (int w = 0; w < W; ++w)
        y[w] = t[w];
    const int rank = rank_of(slot);
    int longest = 0;
    while (any(y)) {
        const int a = lowest(y);
        uint32_t z[W];
#pragma unroll
        for (int w = 0; w < W; ++w)
            z[w] = ~y[w] & span_mask(a, 32 * W - 1, w);
        const int b = lowest(z) - 1;  // last column of the A_8 run
#pragma unroll
        for (int w = 0; w < W; ++w)
            y[w] &= ~span_mask(a, b, w);
        const int e = b + kLong - 1;  // last column of the run of x
        const int L = e - a + 1;
        if (st.nruns >= 0) {
            if (st.nruns < kMaxRuns)
                sk.runs[st.nruns++] = (uint32_t)a | ((uint32_t)e << 8) | ((uint32_t)slot << 16);
            else
                st.nruns = -1;
        }
        longest = max(longest, L);
        if (beats_at(L, rank, a, best_len, best_rank, best_s)) {
            best_len = L;
            best_s = a;
            best_rank = rank;
        }
    }
    return longest;
}

// Solves the range on top of the stack (one call of Algorithm 4's EXEN
// that extracts, or one that finds nothing).  Returns true once the pair is
// finished: its stack is empty, it has made E+1 extractions, or it was
// rejected by the first run's length.
//
// Work is arranged so that the lanes of a warp, each on its own pair, run
// the same instructions: every diagonal first gets the cheap test for a run
// of kLong columns (the same for all lanes), and only the few diagonals that
// have such a run (usually one to three per similar pair, none for most
// dissimilar pairs) get the full ladder, each lane walking its own list.  The
// longest run of each diagonal over all columns is kept from the first
// extraction and bounds it in every later one, where a diagonal that cannot
// beat the best run so far is not examined.
template <int W>
__device__ __forceinline__ bool magnet_step(PairState<W> &st, PairStack &sk, int m)
{
    const uint32_t range = sk.range[--st.sp];
    const int SI = (int)(range & 0xFFu), EI = (int)(range >> 8);
    uint32_t G[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
        G[w] = span_mask(SI, EI, w) & ~st.Nt[w];
    int best_len = 0, best_s = 0, best_rank = kMainRank + 1;
    const bool first = st.done == 0;
    const int range_len = EI - SI + 1;
    // Later extractions: the listed long runs, clipped to the range.
    if (!first && st.nruns > 0) {
        for (int i = 0; i < st.nruns; ++i) {
            const uint32_t r = sk.runs[i];
            const int a = max((int)(r & 0xFFu), SI), e = min((int)((r >> 8) & 0xFFu), EI);
            if (a > e)
                continue;
            const int rank = rank_of((int)(r >> 16));
            if (beats_at(e - a + 1, rank, a, best_len, best_rank, best_s)) {
                best_len = e - a + 1;
                best_s = a;
                best_rank = rank;
            }
        }
    }
    if (W > 2 && !first && st.nruns >= 0 && best_len < kLong && EI < 32 * (SI >> 5) + 64) {
        // A later range inside two words (nearly all of them): the test on
        // the two words only.
        Window win;
        make_window(st, SI, EI, win);
        window_pass<0>(win, st.cand, sk, 0, range_len, best_len, best_s, best_rank);
        for (int j = 1; j <= st.Ep; ++j) {
            window_pass<1>(win, st.cand, sk, j, range_len, best_len, best_s, best_rank);
            window_pass<-1>(win, st.cand, sk, j, range_len, best_len, best_s, best_rank);
        }
    } else if (first || st.nruns < 0 || best_len < kLong) {
        short_pass<W, 0>(st, sk, G, 0, first, range_len, best_len, best_s, best_rank);
        for (int j = 1; j <= st.Ep; ++j) {
            short_pass<W, 1>(st, sk, G, j, first, range_len, best_len, best_s, best_rank);
            short_pass<W, -1>(st, sk, G, j, first, range_len, best_len, best_s, best_rank);
        }
    }
    if (first || st.nruns < 0) {
        for (uint64_t c = st.cand; c; c &= c - 1) {
            const int slot = __ffsll((long long)c) - 1;
            const int rank = rank_of(slot);
            if (!first && !beats(sk.len[slot], rank, best_len, best_rank))
                continue;
            uint32_t x[W];
            build_any(st, G, slot, x);
            if (first && st.nruns >= 0) {
                sk.len[slot] = (uint8_t)list_runs(st, sk, x, slot, best_len, best_s, best_rank);
                continue;
            }
            int s = 0, k = 0;
            // In the first extraction the exact length is kept as the bound
            // for later ones, so it is taken even when it does not win.
            const int L = longest_run(x, rank, first ? 0 : best_len,
                                      first ? kMainRank + 1 : best_rank, s, k);
            if (first)
                sk.len[slot] = (uint8_t)L;
            if (L > 0 && beats(L, rank, best_len, best_rank)) {
                best_len = L;
                best_s = s;
                best_rank = rank;
            }
        }
    }
    if (best_len > 0) {
        if (first && best_len < m / (st.Ep + 1)) {  // ceil((m - E) / (E + 1))
            st.rejected = true;                     // the vector stays all ones
            return true;
        }
        const int e = best_s + best_len - 1;
#pragma unroll
        for (int w = 0; w < W; ++w)
            st.V[w] &= ~span_mask(best_s, e, w);
        ++st.done;
        if (best_s - 2 >= SI)  // left subproblem, solved after the right one
            sk.range[st.sp++] = (uint16_t)(SI | ((best_s - 2) << 8));
        if (e + 2 <= EI)       // right subproblem
            sk.range[st.sp++] = (uint16_t)((e + 2) | (EI << 8));
    }
    return st.sp == 0 || st.done > st.Ep;
}

template <int W>
__device__ __forceinline__ int ones_of(const PairState<W> &st)
{
    int ones = 0;
#pragma unroll
    for (int w = 0; w < W; ++w)
        ones += __popc(st.V[w]);
    return ones;
}

// One warp per group of 32 pairs, one lane per pair; the lanes take their
// extractions in step (first extractions together, then second ones, ...),
// which keeps them on the same code: a lane whose pair is finished waits.
template <int W, bool WITH_N>
__global__ void __launch_bounds__(kMagnetThreads)
magnet_kernel(const FilterArgs a, const int E)
{
    const int lane = threadIdx.x & 31;
    const size_t g = (size_t)blockIdx.x * (kMagnetThreads / 32) + (threadIdx.x >> 5);
    if (g >= groups_of(a.n_pairs))
        return;  // whole warp
    const int m = a.m;
    const size_t pair = g * 32 + lane;
    const bool live = pair < a.n_pairs;
    uint32_t P[6][W];
    load_group<W, WITH_N>(a, g, lane, P);
    PairState<W> st;
    PairStack sk;
    init_pair(st, sk, P, m, a.E_per_pair && live ? min((int)__ldg(a.E_per_pair + pair), E) : E);
    if (live)
        while (!magnet_step(st, sk, m)) {
        }
    const int ones = ones_of(st);
    const uint32_t bits = __ballot_sync(0xFFFFFFFFu, live && ones <= st.Ep);
    if (lane == 0)
        a.accept[g] = bits;
    if (a.count && live)
        a.count[pair] = (uint8_t)ones;
    if (a.vectors) {
        const size_t t = g / kLanes;
        const int l = (int)(g % kLanes);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t col = warp_transpose(live ? st.V[w] : 0u, lane);
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
    const unsigned blocks = (unsigned)((groups + kMagnetThreads / 32 - 1) / (kMagnetThreads / 32));
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
