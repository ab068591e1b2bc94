/*
 * shouji.h -- C ABI of libshouji.so, a GB300 (sm_103a) implementation of the
 * Shouji pre-alignment filter (Alser et al., arXiv 1809.07858).
 *
 * Problem statement (Sec. 2.2 and Algorithm 1 of the paper): for a pair of
 * equal-length sequences, a text T (the reference segment) and a pattern P
 * (the read), and an edit distance threshold E, decide 1 = "similar,
 * alignment needed" or 0 = "dissimilar".  The filter builds the 2E+1
 * diagonal bit-vectors of the neighborhood map (Sec. 2.2.1, Eq. 1), slides
 * a 4-column search window to pick the diagonal segment with the most zeros
 * (Sec. 2.2.2), keeps the chosen segments in the Shouji bit-vector, counts
 * its ones and accepts iff that count is at most E (Sec. 2.2.3).  Results
 * come back one bit per pair, in input order (Sec. 2.3).
 *
 * Conventions shared by every call
 *   - Device pointers are CUDA global memory of the current device, owned by
 *     the caller.  The compute calls never allocate.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous on that stream: a return of
 *     SHOUJI_OK means the work was launched; results are valid once the
 *     stream has reached that point.
 *   - Arguments are checked on the host; a bad one returns SHOUJI_EINVAL and
 *     launches nothing.  A CUDA launch failure returns SHOUJI_ECUDA (the CUDA
 *     error code is kept in shouji_last_cuda_error()).  Nothing aborts, traps
 *     or exits.
 *   - n = 0 pairs is valid and does nothing.
 *   - Bases are the uppercase ASCII letters A, C, G, T and N.  An 'N' never
 *     matches anything, another 'N' included, when its sequence was packed
 *     with an N mask; without one it is read as 'G'.  Other bytes are not
 *     checked: they are read through their bits 1-2 like the four bases.
 *
 * Packed ("bit-sliced") sequence layout, produced by shouji_pack and read by
 * shouji_filter.  Sequences are grouped into tiles of SHOUJI_TILE = 1024 =
 * 32 lanes x 32 bits.  Sequence s lives in tile t = s / 1024, lane
 * l = (s % 1024) / 32, bit b = s % 32.  For position p (0 <= p < m) the
 * base is a 2-bit code (A=00, C=01, G=11, T=10; hi bit, lo bit), stored as
 *     packed[(((size_t)t * m + p) * 32 + l) * 2 + 0]  bit b = hi bit,
 *     packed[(((size_t)t * m + p) * 32 + l) * 2 + 1]  bit b = lo bit,
 * and the optional N mask as
 *     nmask[((size_t)t * m + p) * 32 + l]             bit b = base is 'N'.
 * One 32-bit word thus holds one position of 32 sequences: the filter works
 * on 32 pairs per instruction.  Sizes: shouji_packed_words() and
 * shouji_nmask_words().  Bits of the sequences past n in the last tile are
 * written as zeros.
 */
#ifndef SHOUJI_H
#define SHOUJI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SHOUJI_OK = 0,
    SHOUJI_EINVAL = 1,   /* bad argument; nothing launched */
    SHOUJI_ENOMEM = 2,   /* an allocation failed (pipeline creation only) */
    SHOUJI_ECUDA = 3,    /* a CUDA call failed; see shouji_last_cuda_error() */
    SHOUJI_ETIMEOUT = 4  /* a host wait passed its deadline */
} shouji_status;

#define SHOUJI_TILE 1024 /* sequences per packed tile */
#define SHOUJI_MAX_M 255 /* longest sequence; the per-pair count fits a uint8 */
#define SHOUJI_MAX_E 31  /* largest edit distance threshold (63 diagonals) */

/* Human-readable name of a status code (static storage). */
const char *shouji_status_string(shouji_status s);

/* The cudaError_t of the last failed CUDA call made by this library on the
 * calling host thread (0 when none). */
int shouji_last_cuda_error(void);

/* Number of uint32 words of a packed 2-bit array for n sequences of length
 * m: ceil(n / 1024) * m * 64. */
size_t shouji_packed_words(size_t n, uint32_t m);

/* Number of uint32 words of an N mask for n sequences of length m:
 * ceil(n / 1024) * m * 32. */
size_t shouji_nmask_words(size_t n, uint32_t m);

/*
 * shouji_wait_failures -- how many bounded device waits ran out.
 *
 * Synchronizes the device, writes to *count the number of bounded waits that
 * ran out since the last call (staging waits of shouji_pack, one per CTA that
 * gave up, and hand-over waits of shouji_pack_filter, one per warp group that
 * gave up), and resets that number.  Nonzero means that the output of some
 * launch is incomplete.  No wait runs out in normal operation: the count
 * exists so that a copy that never lands ends the kernel instead of hanging
 * it.
 *   count   host, written.
 * Errors: SHOUJI_EINVAL for NULL count; SHOUJI_ECUDA when the synchronize or
 * the read fails (e.g. an earlier asynchronous error).
 */
shouji_status shouji_wait_failures(uint32_t *count);

/*
 * shouji_selftest_pack_wait -- exercises the path above without a fault.
 *
 * Packs 1024 sequences of 4 bases (one tile: 4 blocks of 256 rows, one CTA
 * each) with every staging copy announced to its mbarrier as 16 bytes longer
 * than it is, so that no wait can complete: each CTA's wait runs out after
 * about a second.  Synchronizes the device and writes to *failures the
 * failures counted by that launch (4); failures counted before the call are
 * discarded.  Takes about a second; the device stays usable.
 *   failures  host, written.
 * Errors: SHOUJI_EINVAL for NULL failures; SHOUJI_ECUDA on a CUDA failure.
 */
shouji_status shouji_selftest_pack_wait(uint32_t *failures);

/*
 * shouji_pack -- ASCII sequences to the packed bit-sliced layout.
 *
 * The FPGA design of the paper compares bases with XOR on an encoded form of
 * the sequences (Sec. 2.3); this call produces the encoded form once, so a
 * set of sequences can be filtered at many thresholds.
 *
 *   seqs    device, n rows of m bytes; row i starts at seqs + i * stride.
 *   stride  bytes between rows, >= m.
 *   n       number of sequences.
 *   m       sequence length, 1 <= m <= SHOUJI_MAX_M.
 *   packed  device, shouji_packed_words(n, m) words (layout above); written.
 *   nmask   device, shouji_nmask_words(n, m) words, or NULL to encode 'N'
 *           as 'G' (no mask).
 * Errors: SHOUJI_EINVAL for NULL seqs/packed (with n > 0), m out of range,
 * stride < m; SHOUJI_ECUDA on a launch failure.
 * Contiguous rows on a 16-byte boundary (stride == m, seqs % 16 == 0) are
 * staged by bulk copies whose completion the kernel waits for with a limit of
 * about one second; a wait that runs out leaves part of `packed` unwritten
 * and is counted for shouji_wait_failures().
 */
shouji_status shouji_pack(const uint8_t *seqs, uint64_t stride, size_t n,
                          uint32_t m, uint32_t *packed, uint32_t *nmask,
                          void *stream);

/*
 * shouji_filter -- the Shouji filter on n_pairs packed pairs (read i =
 * pattern P, reference i = text T, both of length m).
 *
 * Per pair (Sec. 2.2; readings of the paper where it is silent or garbled
 * are fixed as follows): diagonal d in [-E, E] holds at column c the
 * mismatch bit of P[c-d] against T[c] (Eq. 1), 1 outside the band; window c
 * (c = 0..m-1) covers columns c..c+3, columns past the end read as 1; the
 * window's segment is chosen among lower_1, upper_1, ..., lower_E, upper_E
 * by most zeros, a tie going to the first segment that starts with a zero,
 * and the main diagonal replaces the choice only with strictly more zeros;
 * the Shouji bit-vector (all ones at the start) takes the chosen segment
 * only if it has strictly more zeros than the bits it replaces; the pair is
 * accepted iff the vector holds at most E ones.
 *
 *   reads, refs   device, packed (shouji_packed_words(n_pairs, m) words).
 *   reads_nmask,  device N masks of reads and refs (shouji_nmask_words), or
 *   refs_nmask    both NULL.
 *   m             1 <= m <= SHOUJI_MAX_M (the length both were packed with).
 *   n_pairs       number of pairs.
 *   E             0 <= E <= SHOUJI_MAX_E.  With E_per_pair it is the upper
 *                 bound of the per-pair thresholds (the work per pair grows
 *                 with it: 2E+1 diagonals, Eq. 2 of the paper).
 *   E_per_pair    device uint8[n_pairs] with every value <= E, or NULL.
 *                 Values above E are treated as E.
 *   out_accept    device uint32[ceil(n_pairs / 32)]: bit i % 32 of word
 *                 i / 32 = 1 iff pair i is accepted; bits past n_pairs = 0.
 *   out_count     device uint8[n_pairs] = ones in pair i's Shouji bit-vector
 *                 (its edit estimate), or NULL.
 *   out_vectors   device, shouji_nmask_words(n_pairs, m) words, or NULL:
 *                 the Shouji bit-vectors themselves, bit-sliced like an N
 *                 mask (bit b of word ((t*m + c)*32 + l) = column c of pair
 *                 1024t + 32l + b).
 * Errors: SHOUJI_EINVAL for NULL reads/refs/out_accept (with n_pairs > 0),
 * only one N mask given, m or E out of range; SHOUJI_ECUDA on a launch
 * failure.
 */
shouji_status shouji_filter(const uint32_t *reads, const uint32_t *refs,
                            const uint32_t *reads_nmask,
                            const uint32_t *refs_nmask, uint32_t m,
                            size_t n_pairs, int E, const uint8_t *E_per_pair,
                            uint32_t *out_accept, uint8_t *out_count,
                            uint32_t *out_vectors, void *stream);

/*
 * shouji_pack_filter -- shouji_pack of the reads and of the refs followed by
 * shouji_filter (no N masks, one threshold), with the same outputs.
 *
 * When both row sets are contiguous (stride == m) on 16-byte boundaries,
 * E <= 5 and m <= 199, this is one kernel: per SM, 16 warps stream and pack
 * 1024-pair tiles while 8 warps filter the tiles packed before, so the
 * HBM-bound pack and the ALU-bound filter overlap.  Otherwise it launches the
 * two packs and the filter one after the other.
 *
 *   reads, refs    device, n_pairs rows of m ASCII bytes; row i starts at
 *                  reads + i * stride (refs likewise).
 *   stride         bytes between rows, >= m.
 *   n_pairs, m     number of pairs, 1 <= m <= SHOUJI_MAX_M.
 *   E              0 <= E <= SHOUJI_MAX_E.
 *   packed_reads,  device, shouji_packed_words(n_pairs, m) words each, 8-byte
 *   packed_refs    aligned: written with the packed sequences (as
 *                  shouji_pack, 'N' encoded as 'G').
 *   out_accept     device uint32[ceil(n_pairs / 32)], as shouji_filter.
 *   out_count      device uint8[n_pairs], or NULL, as shouji_filter.
 * Errors: SHOUJI_EINVAL for NULL pointers (with n_pairs > 0), misaligned
 * packed arrays, m, stride or E out of range; SHOUJI_ECUDA on a launch
 * failure.  The fused kernel's waits are bounded (about a second) and a wait
 * that runs out is counted for shouji_wait_failures().
 */
shouji_status shouji_pack_filter(const uint8_t *reads, const uint8_t *refs, uint64_t stride,
                                 size_t n_pairs, uint32_t m, int E, uint32_t *packed_reads,
                                 uint32_t *packed_refs, uint32_t *out_accept, uint8_t *out_count,
                                 void *stream);

/*
 * shouji_count -- local and semi-global ("glocal") counting.
 *
 * The paper counts every one of the Shouji bit-vector for end-to-end
 * (global) alignment and leaves out the runs of ones at both ends for local
 * alignment, or at one end for glocal alignment (Sec. 2.2.3; Supplementary
 * Sec. 8, Fig. 6(c), where a 68-base read is filtered against a 100-base
 * reference).  This call recounts Shouji bit-vectors written by
 * shouji_filter (out_vectors) under a count mode:
 *   SHOUJI_COUNT_GLOBAL        every one (the count of shouji_filter);
 *   SHOUJI_COUNT_LOCAL         not the runs of ones at the two ends;
 *   SHOUJI_COUNT_GLOCAL_START  not the run of ones at the start;
 *   SHOUJI_COUNT_GLOCAL_END    not the run of ones at the end.
 * A vector with no zero counts m in every mode.  A read shorter than its
 * reference is filtered by packing it padded with 'N' to the reference
 * length, with N masks: an 'N' matches nothing, like the cells past the end
 * of the read in the paper's map.
 *
 *   vectors      device, bit-sliced Shouji bit-vectors of n_pairs pairs of
 *                length m (out_vectors of shouji_filter, or the MAGNET
 *                bit-vectors of shouji_magnet).
 *   E, E_per_pair as shouji_filter (the accept threshold).
 *   mode         one of the four modes above.
 *   out_accept   device uint32[ceil(n_pairs / 32)]: count <= E.
 *   out_count    device uint8[n_pairs] or NULL: the count under the mode.
 * Errors: SHOUJI_EINVAL for NULL vectors/out_accept (with n_pairs > 0), m, E
 * or mode out of range; SHOUJI_ECUDA on a launch failure.
 */
#define SHOUJI_COUNT_GLOBAL 0
#define SHOUJI_COUNT_LOCAL 1
#define SHOUJI_COUNT_GLOCAL_START 2
#define SHOUJI_COUNT_GLOCAL_END 3

shouji_status shouji_count(const uint32_t *vectors, uint32_t m, size_t n_pairs,
                           int E, const uint8_t *E_per_pair, int mode,
                           uint32_t *out_accept, uint8_t *out_count,
                           void *stream);

/*
 * shouji_magnet -- the MAGNET filter (Supplementary Sec. 7, Algorithms 3
 * and 4 of the paper) on the same packed pairs and the same neighborhood
 * map as shouji_filter.
 *
 * Per pair: the MAGNET bit-vector starts as all ones.  An extraction takes,
 * inside the current column range, the longest run of zeros over the 2E+1
 * diagonals, writes it as zeros into the vector, and keeps the column just
 * before and just after it out of both subranges (encapsulation); the
 * subrange right of the run is solved first, with all of its own
 * subranges, then the subrange left of it.  There are at most E+1
 * extractions, and a range without a zero extracts nothing.  If the first
 * run is shorter than ceil((m-E)/(E+1)) columns the pair is rejected with
 * the vector left all ones.  Ties between equally long runs go to upper_1,
 * lower_1, upper_2, lower_2, ... in that order, to the main diagonal only
 * when no other diagonal has a run that long, and within a diagonal to the
 * leftmost run.  The pair is accepted iff the vector holds at most E ones.
 *
 * Arguments, layouts and errors are those of shouji_filter; out_vectors
 * receives the MAGNET bit-vectors in the bit-sliced layout of an N mask,
 * which shouji_count recounts for local and glocal alignment.
 */
shouji_status shouji_magnet(const uint32_t *reads, const uint32_t *refs,
                            const uint32_t *reads_nmask,
                            const uint32_t *refs_nmask, uint32_t m,
                            size_t n_pairs, int E, const uint8_t *E_per_pair,
                            uint32_t *out_accept, uint8_t *out_count,
                            uint32_t *out_vectors, void *stream);

/*
 * shouji_compact_workspace_size -- bytes of device workspace that
 * shouji_compact needs for n_pairs pairs (0 for n_pairs = 0).
 */
size_t shouji_compact_workspace_size(size_t n_pairs);

/*
 * shouji_compact -- indices of the accepted pairs, in input order.
 *
 * The paper's accelerator returns one result bit per pair in input order
 * and the host picks the survivors (Sec. 2.3); this call does that
 * selection on the device.
 *
 *   accept      device uint32[ceil(n_pairs / 32)], as written by
 *               shouji_filter (bits past n_pairs are ignored).
 *   n_pairs     number of pairs, < 2^32.
 *   out_idx     device uint32[n_pairs] (worst case); the first *out_n
 *               entries receive the accepted pair indices in increasing order.
 *   out_n       device uint32[1]: number of accepted pairs.
 *   workspace   device scratch of at least workspace_bytes >=
 *               shouji_compact_workspace_size(n_pairs) bytes, 16-byte
 *               aligned; its contents on entry do not matter.
 * Errors: SHOUJI_EINVAL for NULL pointers (with n_pairs > 0), n_pairs >=
 * 2^32, a short or misaligned workspace; SHOUJI_ECUDA on a launch failure.
 */
shouji_status shouji_compact(const uint32_t *accept, size_t n_pairs,
                             uint32_t *out_idx, uint32_t *out_n,
                             void *workspace, size_t workspace_bytes,
                             void *stream);

/*
 * shouji_compact_noalloc -- shouji_compact without a caller-supplied
 * workspace.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc, such as a program whose device memory
 * is entirely owned by another allocator with a fixed budget, or a
 * latency-bound loop that must not call cudaMalloc/cudaFree because they can
 * synchronize the device.  It allocates nothing and calls no allocating
 * routine.
 *
 * Its workspace is a fixed 64 KB __device__ array inside libshouji.so, held
 * on every GPU that loads the library until the process exits.  The first
 * call on each device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  Every call on a device shares the one array:
 * two calls whose work overlaps on the GPU (e.g. on two streams) race and
 * may return wrong indices; serialize them.  The array keeps the last
 * call's contents, and nothing in it needs to start at zero.
 *
 *   accept, n_pairs, out_idx, out_n, stream: as shouji_compact.
 * Errors: SHOUJI_EINVAL for n_pairs > SHOUJI_NOALLOC_MAX_PAIRS (2^29) or
 * NULL pointers (with n_pairs > 0); SHOUJI_ECUDA on a failed address lookup
 * or launch.
 */
#define SHOUJI_NOALLOC_MAX_PAIRS ((size_t)1 << 29)

shouji_status shouji_compact_noalloc(const uint32_t *accept, size_t n_pairs,
                                     uint32_t *out_idx, uint32_t *out_n,
                                     void *stream);

/*
 * Host pipeline -- the whole filter for pairs held in HOST memory.
 *
 * The paper's accelerator receives pairs from the host and returns one
 * result bit per pair in input order (Sec. 2.3); this object does the same
 * on a GPU: it cuts a batch into chunks and alternates two CUDA streams so
 * that the host-to-device copy of one chunk overlaps the pack, filter and
 * compaction of the previous one.
 *
 * shouji_pipeline_create allocates every device buffer the runs need on the
 * current device (two chunk slots, an index array for max_pairs survivors)
 * and the two streams.
 *   m            sequence length, 1 <= m <= SHOUJI_MAX_M.
 *   chunk_pairs  pairs per chunk (> 0; rounded up to a multiple of 1024).
 *   max_pairs    largest n_pairs whose survivor indices a run may return
 *                (< 2^32; 0 = runs return no indices).
 *   with_n       nonzero: 'N' bases match nothing (N masks are built).
 *   out          receives the pipeline; NULL on failure.
 * Errors: SHOUJI_EINVAL, SHOUJI_ENOMEM (nothing is leaked), SHOUJI_ECUDA.
 *
 * shouji_pipeline_run filters n_pairs pairs and returns when all results
 * are in host memory (it synchronizes its own streams only).  Host buffers
 * should be pinned (cudaHostAlloc) for the copies to overlap.
 *   reads, refs  host, n_pairs rows of m bytes, row i at + i * stride.
 *   E            0 <= E <= SHOUJI_MAX_E.
 *   accept       host uint32[ceil(n_pairs / 32)] (layout of shouji_filter).
 *   count        host uint8[n_pairs] or NULL.
 *   idx          host uint32[n_pairs] or NULL: survivor indices, in order
 *                (needs n_pairs <= max_pairs).
 *   n_accepted   host, or NULL: number of accepted pairs.
 * Errors: SHOUJI_EINVAL (bad argument, nothing launched), SHOUJI_ECUDA.
 *
 * shouji_pipeline_destroy frees everything (NULL is a no-op).  A pipeline
 * must not be used by two host threads at once.
 */
typedef struct shouji_pipeline shouji_pipeline;

shouji_status shouji_pipeline_create(uint32_t m, size_t chunk_pairs,
                                     size_t max_pairs, int with_n,
                                     shouji_pipeline **out);

shouji_status shouji_pipeline_run(shouji_pipeline *pipeline,
                                  const uint8_t *reads, const uint8_t *refs,
                                  uint64_t stride, size_t n_pairs, int E,
                                  uint32_t *accept, uint8_t *count,
                                  uint32_t *idx, uint64_t *n_accepted);

void shouji_pipeline_destroy(shouji_pipeline *pipeline);

/*
 * Batched filter -- pairs of mixed lengths and thresholds in one launch.
 *
 * The work per pair grows with m (2E + 2) (Eq. 2 of the paper), and the
 * 32 pairs that share a bit-sliced group cost as much as their longest,
 * most tolerant member.  A batch object therefore buckets each batch on the
 * device by (m, E), packs every bucket, runs one persistent filter kernel per
 * threshold over all of its buckets and gathers the results back to input
 * order.  The whole sequence is captured once into a CUDA graph; every run
 * is one graph launch.  The global mode of the paper applies: a pair's read
 * and reference have the same length (Supp. Sec. 8).
 *
 * shouji_batch_create allocates every device buffer on the current device.
 *   max_pairs    largest batch (< 2^31).
 *   max_m        longest sequence, <= SHOUJI_MAX_M.
 *   e_min, e_max thresholds the batches may use (0 <= e_min <= e_max <= 31);
 *                one filter kernel per threshold in the range is in the graph.
 *   with_n       nonzero: 'N' matches nothing (N masks are built).
 *   tune_cache   path of a tuning cache written by shouji_batch_tune, or NULL
 *                (defaults: 128 threads, 4 CTAs per SM, strided schedule).
 * Errors: SHOUJI_EINVAL, SHOUJI_ENOMEM (nothing leaked), SHOUJI_ECUDA.
 *
 * shouji_batch_run filters one batch, asynchronously on `stream`.  Device
 * pointers:
 *   reads, refs   n_pairs rows, row i at + i * stride, lens[i] bases each;
 *                 each buffer must be readable for n_pairs * stride bytes
 *                 (whole 16-byte chunks are read when stride is a multiple of
 *                 16 no smaller than max_m rounded up to 16).
 *   lens          uint16[n_pairs], each in [1, max_m].
 *   E_per_pair    uint8[n_pairs], each in [e_min, e_max].
 *   out_accept    uint32[ceil(n_pairs / 32)] (layout of shouji_filter).
 *   out_count     uint8[n_pairs] or NULL.
 * A pair whose length or threshold is out of range is rejected (accept 0,
 * count 255) and counted by shouji_batch_invalid.  Before it writes a new
 * argument block, a run waits until the previous run of the same object has
 * started on the GPU; one object runs one batch at a time, and concurrent
 * batches need one object each.
 * Errors: SHOUJI_EINVAL (nothing launched), SHOUJI_ECUDA.
 *
 * shouji_batch_invalid waits for the last run and returns its number of
 * rejected out-of-range pairs.
 *
 * shouji_batch_tune is the autotuner.  It runs the bucketing and packing of
 * the given batch, then times every launch shape of each threshold's filter
 * kernel (CTA of 64 or 128 threads, 1-8 CTAs per SM; groups grid-strided,
 * in a contiguous range per CTA, or taken from a shared counter) and keeps
 * the fastest.  It appends them to tune_cache
 * (when not NULL) as "<gpu> <E> <threads> <ctas/SM> <schedule> <ms>" lines,
 * which shouji_batch_create reads back.  It does not write out_accept /
 * out_count: call shouji_batch_run afterwards.  It synchronizes `stream`.
 *
 * shouji_batch_destroy waits for the last run and frees everything.
 */
typedef struct shouji_batch shouji_batch;

shouji_status shouji_batch_create(size_t max_pairs, uint32_t max_m, int e_min,
                                  int e_max, int with_n, const char *tune_cache,
                                  shouji_batch **out);

shouji_status shouji_batch_run(shouji_batch *batch, const uint8_t *reads,
                               const uint8_t *refs, uint64_t stride,
                               const uint16_t *lens, const uint8_t *E_per_pair,
                               size_t n_pairs, uint32_t *out_accept,
                               uint8_t *out_count, void *stream);

shouji_status shouji_batch_invalid(shouji_batch *batch, uint64_t *n_invalid);

shouji_status shouji_batch_tune(shouji_batch *batch, const uint8_t *reads,
                                const uint8_t *refs, uint64_t stride,
                                const uint16_t *lens, const uint8_t *E_per_pair,
                                size_t n_pairs, uint32_t *out_accept,
                                uint8_t *out_count, const char *tune_cache,
                                void *stream);

void shouji_batch_destroy(shouji_batch *batch);

/*
 * Serving loop -- filter requests as they arrive (continuous batching).
 *
 * The paper integrates the filter into read mappers, which produce candidate
 * pairs continuously and keep only the pairs the filter accepts (Sec. 3.6,
 * Table 15).  A server takes requests from any host thread.  A dispatcher
 * thread admits them in arrival order into slots.  A slot is a batch object
 * (one CUDA graph) with its own stream and device buffers.  An admitted
 * request is copied in, filtered and copied out on its slot's stream, so
 * requests admitted while others are on the GPU run concurrently with them;
 * a finished slot takes the next queued request at once.
 *
 * shouji_server_create makes slots on the current device until the next
 * one would exceed memory_budget bytes (the first slot measures the cost of
 * one) or max_slots exist, then starts the dispatcher.
 *   max_request_pairs  largest request; max_m, e_min, e_max, with_n,
 *                      tune_cache: as shouji_batch_create.
 *   max_stride         largest row stride of a request (>= max_m).
 * Errors: SHOUJI_EINVAL; SHOUJI_ENOMEM (not even one slot fits the budget
 * or the device); SHOUJI_ECUDA.
 *
 * shouji_server_info: number of slots and device bytes of one slot.
 *
 * shouji_server_submit queues one request and returns at once with its id.
 * Host buffers, as shouji_batch_run's device ones (reads/refs rows of
 * `stride` bytes, lens, E_per_pair, accept, optional count), must stay
 * valid and untouched until shouji_server_wait returns for the id.  Pinned
 * host buffers let the copies run asynchronously.
 * Errors: SHOUJI_EINVAL (bad argument or the server is stopping).
 *
 * shouji_server_wait blocks until the request is done or timeout_s seconds
 * have passed (SHOUJI_ETIMEOUT; the request stays queued or in flight and
 * can be waited for again).  On completion it writes the latency, from
 * submit to completion in seconds, into latency_s (when not NULL), forgets
 * the id, and returns the request's status.
 *
 * shouji_server_destroy finishes every queued and in-flight request, stops
 * the dispatcher and frees everything.
 */
typedef struct shouji_server shouji_server;

shouji_status shouji_server_create(size_t max_request_pairs, uint32_t max_m,
                                   uint64_t max_stride, int e_min, int e_max,
                                   int with_n, size_t memory_budget,
                                   int max_slots, const char *tune_cache,
                                   shouji_server **out);

shouji_status shouji_server_info(shouji_server *server, int *slots,
                                 uint64_t *bytes_per_slot);

shouji_status shouji_server_submit(shouji_server *server, const uint8_t *reads,
                                   const uint8_t *refs, uint64_t stride,
                                   const uint16_t *lens,
                                   const uint8_t *E_per_pair, size_t n_pairs,
                                   uint32_t *accept, uint8_t *count,
                                   uint64_t *request_id);

shouji_status shouji_server_wait(shouji_server *server, uint64_t request_id,
                                 double timeout_s, double *latency_s);

void shouji_server_destroy(shouji_server *server);

#ifdef __cplusplus
}
#endif

#endif /* SHOUJI_H */
