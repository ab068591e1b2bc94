// Batched filter for pairs of mixed lengths and thresholds.
//
// The cost of a pair is proportional to m (2E + 2) (Eq. 2 of the paper), and
// a bit-sliced group of 32 pairs costs as much as its longest, most tolerant
// member.  So the batch is first bucketed on the device by (m, E): buckets
// are laid out by m (each m-class starts on a 1024-pair tile, because a
// packed tile has one length) and, inside an m-class, by E (each bucket
// starts on a 32-pair group, because a group runs one threshold).  The
// pairs are packed bucket by bucket, every threshold class is filtered by a
// persistent kernel specialised for its E that walks all of its buckets, and
// the counts are gathered back to input order.
#pragma once

#include "shouji_internal.cuh"

namespace shouji {
namespace batch {

constexpr int kMaxM = 256;            // lengths 1..255
constexpr int kMaxE = 32;             // thresholds 0..31
constexpr int kBins = kMaxM * kMaxE;  // bucket key = m * 32 + E
constexpr uint16_t kBadKey = 0xFFFF;
constexpr uint32_t kNoPair = 0xFFFFFFFFu;
// Windows per chunk of the filter's loop that the tuner may choose per
// threshold: 4 always, 8 for thresholds up to kMaxE8 (the longer chunk keeps
// about twice the map columns live; above that its registers grow past 200).
constexpr int kMaxE8 = 6;

// Per-run arguments, read by every kernel from device memory (the CUDA graph
// copies them from a pinned host block at the start of each launch).
struct Args {
    const uint8_t *reads, *refs;
    uint64_t stride;
    // null: the reference of pair i is the row refs + i * stride; else it
    // starts at refs + ref_off[i] (a reference text kept on the device)
    const uint64_t *ref_off;
    const uint16_t *lens;
    const uint8_t *E_per_pair;
    uint64_t n;
    uint32_t *accept;
    uint8_t *count;
};

// Bucket layout of one run, computed on the device.
struct Tables {
    uint32_t bin_slot[kBins];   // first slot of bucket (m, E)
    uint32_t n_mc;              // number of m-classes
    uint32_t mc_m[kMaxM];       // length of m-class c
    uint32_t mc_slot[kMaxM];    // first slot of m-class c (multiple of 1024)
    uint64_t mc_poff[kMaxM];    // offset of its packed tiles, in uint2 units
    uint32_t mc_block[kMaxM + 1];  // prefix of pack blocks (256 slots each)
    uint32_t total_slots;
    uint32_t ec_first[kMaxE], ec_count[kMaxE], ec_groups[kMaxE];
    // buckets of threshold E at [E * kMaxM, E * kMaxM + ec_count[E]), by m
    uint32_t bk_m[kBins], bk_slot[kBins], bk_count[kBins], bk_gstart[kBins], bk_mc[kBins];
    uint32_t n_invalid;         // pairs with a length or threshold out of range
    uint32_t work[kMaxE];       // next group of each threshold (dynamic schedule)
};

// Arguments of the persistent filter kernel of one threshold.
struct FilterParams {
    const Tables *tables;
    const uint2 *preads, *prefs;
    const uint32_t *nreads, *nrefs;  // N masks or null
    uint8_t *count_slot;             // counts in slot order
    uint32_t *work;                  // Tables::work (dynamic schedule)
    int schedule;                    // 0: grid-strided groups; 1: a contiguous range per
                                     // CTA; 2: CTAs take blockDim groups at a time from a
                                     // shared counter
    int u;                           // windows per chunk: 4, or 8 for small thresholds
};

template <int E>
cudaError_t launch_filter_E(const FilterParams &p, int threads, int ctas, cudaStream_t s);

}  // namespace batch
}  // namespace shouji
