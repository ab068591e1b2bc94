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
 *     with an N mask.  Without one it is read as 'G', which gives other
 *     results; every pack without an N mask therefore looks for 'N' bytes
 *     on the device: shouji_unmasked_n() returns SHOUJI_EINVAL once
 *     shouji_pack, shouji_pack_filter or the batched and served forms
 *     without with_n have seen one, and shouji_pipeline_run without with_n
 *     returns SHOUJI_EINVAL itself.  Other bytes are read
 *     through their bits 1-2 like the four bases (a byte with bit 3 set,
 *     such as 'n', is reported like an 'N').
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
 * shouji_unmasked_n -- whether a pack without an N mask read an 'N'.
 *
 * The paper's filter compares bases (Eq. 1); an 'N' (an unknown base) is read
 * here as matching nothing, another 'N' included, which needs an N mask
 * (shouji_pack with nmask, shouji_filter with both masks, the batched and
 * served forms and the host pipeline with with_n).  Without a mask an 'N' has
 * no 2-bit code of its own and is read as 'G'.  So that such results are
 * never taken silently, every pack without a mask (shouji_pack,
 * shouji_pack_filter, the batched and served forms without with_n) checks
 * its bytes on the device and sets a flag when one holds an 'N'.  This call synchronizes the
 * device, writes the flag to *seen (1: at least one pack without an N mask
 * since the last call read an 'N', so its pairs' results differ from the
 * masked ones; 0: none did), resets it, and returns SHOUJI_EINVAL when it was
 * set.  The flag is shared by all calls of the process on the device: read
 * it after the calls whose input is in question, with no other unmasked
 * pack running.  shouji_pipeline_run (with_n = 0) keeps a flag per pipeline
 * instead and reports through its own status.
 *   seen   host, written.
 * Errors: SHOUJI_EINVAL for NULL seen, and when the flag was set;
 * SHOUJI_ECUDA when the synchronize or the read fails.
 */
shouji_status shouji_unmasked_n(int *seen);

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
 * shouji_alu_probe -- measured issue rate of one integer instruction kind.
 *
 * The filter of Sec. 2.2 is computed here as bit-sliced integer logic, 32
 * pairs per instruction, so its roofline is the issue rate of the GPU's
 * integer pipes, not a memory or tensor figure.  This call measures that rate on
 * the current device: one CTA of 1024 threads per SM runs independent
 * dependency chains of the chosen instruction, and each CTA counts its own
 * SM cycles around the loop.  The result, in lane-operations per SM clock,
 * does not depend on the clock the GPU runs at; multiplied by the SM count
 * and the maximum SM clock it gives the peak rate.
 *   op    SHOUJI_PROBE_LOP3 (3-input logic), _SHF (funnel shift), _PRMT
 *         (byte permute), _IADD3 (3-input add), _IMAD (integer
 *         multiply-add), _POPC (population count), or _LOP3_IMAD (half of
 *         the chains LOP3, half IMAD: the combined rate of two pipes).
 *   lane_ops_per_sm_clock  host, written: median over the SMs.
 * Unlike the compute calls, this one allocates two small device buffers
 * (freed before it returns) and synchronizes the device.  It takes a few
 * milliseconds.
 * Errors: SHOUJI_EINVAL for a NULL output or an unknown op; SHOUJI_ECUDA on
 * a CUDA failure.
 */
#define SHOUJI_PROBE_LOP3 0
#define SHOUJI_PROBE_SHF 1
#define SHOUJI_PROBE_PRMT 2
#define SHOUJI_PROBE_IADD3 3
#define SHOUJI_PROBE_IMAD 4
#define SHOUJI_PROBE_POPC 5
#define SHOUJI_PROBE_LOP3_IMAD 6

shouji_status shouji_alu_probe(int op, double *lane_ops_per_sm_clock);

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
 *                  shouji_pack without a mask: 'N' read as 'G', and
 *                  flagged for shouji_unmasked_n).
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
 * shouji_pack_filter_fused -- whether shouji_pack_filter with these
 * arguments runs as the one fused kernel (1) or as separate pack and filter
 * launches (0).  Both give the same results; the query exists so that a
 * caller (or a benchmark) can tell which kernel it is timing.  The answer
 * depends on the row layout, m, E and on the compiled kernel itself (its
 * register split needs an exact register count), so it needs the device.
 *   reads, refs, stride, m, E  as shouji_pack_filter (nothing is read).
 *   fused   host, written.
 * Errors: SHOUJI_EINVAL for NULL fused or m, stride or E out of range;
 * SHOUJI_ECUDA when the kernel's attributes cannot be read.
 */
shouji_status shouji_pack_filter_fused(const uint8_t *reads, const uint8_t *refs,
                                       uint64_t stride, uint32_t m, int E, int *fused);

/*
 * shouji_pack_filter_results -- shouji_pack_filter for a caller that wants
 * only the results (accept bits and counts), not the packed sequences: the
 * filter of Sec. 2.2 on ASCII pairs, with the same results.
 *
 * Where the fused kernel applies (shouji_pack_filter_fused gives 1), each
 * CTA packs its tiles into a ring of its own in the workspace: the tile of
 * hand-over slot q goes to ring entry q, over the tile that used the slot
 * before (the producers wait until it has been filtered).  The rings of all
 * CTAs take about 93 MB at m = 100, which stays in L2, so the packed words
 * need not reach HBM.  Otherwise the workspace holds both packed arrays and
 * the call is shouji_pack_filter.
 *
 *   reads, refs, stride, n_pairs, m, E   as shouji_pack_filter.
 *   workspace   device, 16-byte aligned, at least the bytes that
 *               shouji_pack_filter_workspace_size gives for the same
 *               arguments on the current device; its contents are scratch.
 *   out_accept, out_count                as shouji_pack_filter.
 * Errors: SHOUJI_EINVAL for NULL pointers (with n_pairs > 0), a short or
 * misaligned workspace, m, stride or E out of range; SHOUJI_ECUDA on a
 * launch failure.  Bounded waits as shouji_pack_filter.
 *
 * shouji_pack_filter_workspace_size writes that size to *bytes (0 for
 * n_pairs = 0): 2 * 12 tiles * 256 m bytes per CTA of the fused kernel
 * (one per SM, at most one per 1024-pair tile), else
 * 2 * 4 * shouji_packed_words(n_pairs, m).  Errors: SHOUJI_EINVAL for NULL
 * bytes or m, stride or E out of range; SHOUJI_ECUDA when the device cannot
 * be queried.
 */
shouji_status shouji_pack_filter_workspace_size(const uint8_t *reads, const uint8_t *refs,
                                                uint64_t stride, size_t n_pairs, uint32_t m,
                                                int E, size_t *bytes);

shouji_status shouji_pack_filter_results(const uint8_t *reads, const uint8_t *refs,
                                         uint64_t stride, size_t n_pairs, uint32_t m, int E,
                                         void *workspace, size_t workspace_bytes,
                                         uint32_t *out_accept, uint8_t *out_count,
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
 * in every CUDA context that loads the library's kernels until that context
 * is destroyed (for the primary context: until the process exits or the
 * device is reset).  The array's device address belongs to a context, so the
 * first call in each context (the primary context of a device, a new one
 * after cudaDeviceReset, or a context the program created with the driver
 * API) looks it up (cudaGetSymbolAddress) with that context current and
 * caches it under the context's id; make that first call before any stream
 * capture.  Every call in a context shares the one array: two calls whose
 * work overlaps on the GPU (e.g. on two streams) race and may return wrong
 * indices; serialize them.  The array keeps the last call's contents, and
 * nothing in it needs to start at zero.
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
 * should be pinned (cudaHostAlloc) for the copies to overlap.  A pipeline
 * created without with_n keeps a flag of its own, like the one of
 * shouji_unmasked_n, and returns SHOUJI_EINVAL, with every result written,
 * when one of the run's sequences held an 'N' (read as 'G').
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

/*
 * shouji_pipeline_run_packed is shouji_pipeline_run for pairs that the
 * caller holds in the packed layout described at the top of this header
 * (for example written by shouji_pack and kept): the copies carry 2 bits per
 * base instead of 8, and no pack runs on the device.
 *   reads, refs      host uint32[shouji_packed_words(n_pairs, m)] each.
 *   reads_n, refs_n  host uint32[shouji_nmask_words(n_pairs, m)] each: the N
 *                    masks, or both NULL (no base is 'N').  Masks need a
 *                    pipeline created with with_n.
 *   the rest         as for shouji_pipeline_run.
 * Errors: SHOUJI_EINVAL (bad argument, only one mask, masks without with_n;
 * nothing launched), SHOUJI_ECUDA.  Bits past n_pairs in the last tile are
 * read but their results are not returned.
 */
shouji_status shouji_pipeline_run_packed(shouji_pipeline *pipeline,
                                         const uint32_t *reads, const uint32_t *refs,
                                         const uint32_t *reads_n, const uint32_t *refs_n,
                                         size_t n_pairs, int E, uint32_t *accept,
                                         uint8_t *count, uint32_t *idx,
                                         uint64_t *n_accepted);

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
 * count 255) and counted by shouji_batch_invalid.  The object holds two
 * argument blocks, each with its own captured graph, and alternates between
 * them: a run waits only for the run two before it (which used the same
 * block) to have finished, so the host can queue a run while the previous
 * one is still on the GPU.  All runs of one object share its device
 * buffers: queue them on one stream (they then run one after the other);
 * concurrent batches need one object each.
 * Errors: SHOUJI_EINVAL (nothing launched), SHOUJI_ECUDA.
 *
 * shouji_batch_invalid waits for the last run and returns its number of
 * rejected out-of-range pairs.
 *
 * shouji_batch_timing waits for the last run and writes the durations, in
 * milliseconds, that the graph itself recorded (event nodes between its
 * stages): ms[0] the whole graph, ms[1] bucketing (classify, scan, fill,
 * scatter), ms[2] the gather-pack, ms[3] the filters (all thresholds, from
 * the fork to the last join), ms[4] finalize, and ms[5 + E] the filter
 * kernel of threshold E alone (-1 for thresholds outside [e_min, e_max], and
 * everywhere before the first run).  n must be at least SHOUJI_BATCH_TIMES.
 *
 * shouji_batch_tune is the autotuner.  It runs the bucketing and packing of
 * the given batch, then times every launch shape of each threshold's filter
 * kernel (CTA of 64 or 128 threads, 1-8 CTAs per SM; groups grid-strided,
 * in a contiguous range per CTA, or taken from a shared counter; 4 or, for
 * E <= 6, 8 windows per chunk of the filter's inner loop) and keeps the
 * fastest.  It appends them to tune_cache (when not NULL) as
 * "<gpu> <E> <threads> <ctas/SM> <schedule> <windows> <ms>" lines, which
 * shouji_batch_create reads back; shouji_batch_shape returns the shape a
 * threshold's kernel runs with.  It does not write out_accept /
 * out_count: call shouji_batch_run afterwards.  It synchronizes `stream`.
 *
 * shouji_batch_destroy waits for the last run and frees everything.
 */
typedef struct shouji_batch shouji_batch;

shouji_status shouji_batch_create(size_t max_pairs, uint32_t max_m, int e_min,
                                  int e_max, int with_n, const char *tune_cache,
                                  shouji_batch **out);

/* Device bytes that shouji_batch_create with these arguments allocates (0
 * for arguments it would reject); for planning device memory. */
size_t shouji_batch_device_bytes(size_t max_pairs, uint32_t max_m, int e_min, int e_max,
                                 int with_n);

shouji_status shouji_batch_run(shouji_batch *batch, const uint8_t *reads,
                               const uint8_t *refs, uint64_t stride,
                               const uint16_t *lens, const uint8_t *E_per_pair,
                               size_t n_pairs, uint32_t *out_accept,
                               uint8_t *out_count, void *stream);

/*
 * shouji_batch_run_at -- shouji_batch_run with the references taken from a
 * text kept on the device (e.g. a reference genome loaded once): pair i
 * compares read i (row reads + i * stride) with the lens[i] bytes of
 * ref_text starting at ref_offsets[i] (device uint64[n_pairs]; any byte
 * offset, ref_offsets[i] + lens[i] within the text).  In a read mapper the
 * candidate locations of a read are offsets into the reference (Sec. 3.6 of
 * the paper filters the candidate pairs a mapper produces); the references
 * then need no copy per batch.  Everything else is as shouji_batch_run.
 */
shouji_status shouji_batch_run_at(shouji_batch *batch, const uint8_t *reads, uint64_t stride,
                                  const uint8_t *ref_text, const uint64_t *ref_offsets,
                                  const uint16_t *lens, const uint8_t *E_per_pair,
                                  size_t n_pairs, uint32_t *out_accept, uint8_t *out_count,
                                  void *stream);

shouji_status shouji_batch_invalid(shouji_batch *batch, uint64_t *n_invalid);

shouji_status shouji_batch_shape(shouji_batch *batch, int E, int *threads, int *ctas_per_sm,
                                 int *schedule, int *windows);

#define SHOUJI_BATCH_TIMES (5 + SHOUJI_MAX_E + 1)

shouji_status shouji_batch_timing(shouji_batch *batch, float *ms, int n);

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
 * Table 15).  A server takes requests from any host thread; a dispatcher
 * thread admits them in arrival order by device memory.  A worker is a
 * batch object (one CUDA graph per run) with its own stream and staging
 * buffers, sized for a capacity class of 4096 x 2^k pairs (the last class is
 * max_request_pairs).  A request runs on the smallest free worker that holds
 * it; when none is free, a worker of its class is made if it fits in the
 * memory budget next to everything already held (idle workers are released,
 * least recently used first, to make room), and otherwise the request waits
 * for a running one to finish.  A request thus holds device memory in
 * proportion to its size, and requests admitted while others are on the GPU
 * run concurrently with them.  Making or releasing a worker allocates or
 * frees device memory, which can briefly synchronize the device.
 *
 * shouji_server_create starts the dispatcher; workers are made on demand.
 *   max_request_pairs  largest request (< 2^31); max_m, e_min, e_max, with_n,
 *                      tune_cache: as shouji_batch_create.
 *   max_stride         largest row stride of a request (>= max_m).
 *   memory_budget      device bytes the server may hold (workers and
 *                      resident references).
 *   max_slots          most workers at once (requests on the GPU at once).
 * Errors: SHOUJI_EINVAL; SHOUJI_ENOMEM (the budget cannot hold one worker
 * for max_request_pairs); SHOUJI_ECUDA.
 *
 * shouji_server_info: number of workers held now, and device bytes of a
 * worker for max_request_pairs.  shouji_server_stats_read: the memory and
 * admission counters below.
 *
 * shouji_server_add_reference copies a reference text (any bytes, e.g. a
 * chromosome in ASCII) to the device, where it stays until the server is
 * destroyed, counted against the budget; writes its id.  Requests then name
 * their reference segments by offset into it instead of sending them.
 * Errors: SHOUJI_EINVAL; SHOUJI_ENOMEM when it would leave no room for one
 * worker of the largest class; SHOUJI_ECUDA.
 *
 * shouji_server_submit_request queues one request and returns at once with
 * its id.  The request (copied) names:
 *   reads          host rows of the reads, row i at reads + i * stride;
 *   refs           host rows of the reference segments (same stride), or
 *                  NULL to take pair i's segment from the resident text
 *                  ref_id at byte ref_offsets[i] (host uint64[n_pairs]; every
 *                  segment must lie inside the text, else SHOUJI_EINVAL);
 *   lens, E_per_pair, n_pairs  host arrays and count, as shouji_batch_run;
 *   accept, count  outputs (layout of shouji_filter; count may be NULL):
 *                  host memory, or device memory of the server's device with
 *                  SHOUJI_SERVE_DEVICE_RESULTS in flags (written by the
 *                  filter directly, no copy back).
 * Host buffers must stay valid and untouched until the request is waited
 * for.  Pinned host buffers let the copies run asynchronously; results for
 * host buffers that are not pinned go through pinned staging of the
 * worker's and are copied over when the request completes.
 * shouji_server_submit is the same for host rows of reads and references.
 * Errors: SHOUJI_EINVAL (bad argument or the server is stopping).
 *
 * shouji_server_wait blocks until the request is done or timeout_s seconds
 * have passed (SHOUJI_ETIMEOUT; the request stays queued or in flight and
 * can be waited for again).  On completion it writes the latency, from
 * submit to completion in seconds, into latency_s (when not NULL), forgets
 * the id, and returns the request's status.  shouji_server_wait_timed also
 * writes times[1] and times[2]: when the request's work started and ended on
 * the GPU, in seconds since the server was created (CUDA events around its
 * copies and its graph), from which the overlap of requests on the device
 * can be measured; times[0] is the latency.
 *
 * shouji_server_destroy finishes every queued and in-flight request, stops
 * the dispatcher and frees everything.
 */
typedef struct shouji_server shouji_server;

#define SHOUJI_SERVE_DEVICE_RESULTS 1

typedef struct {
    const uint8_t *reads;
    const uint8_t *refs;
    uint64_t stride;
    uint32_t ref_id;
    const uint64_t *ref_offsets;
    const uint16_t *lens;
    const uint8_t *E_per_pair;
    size_t n_pairs;
    uint32_t *accept;
    uint8_t *count;
    int flags;
} shouji_server_request;

typedef struct {
    uint64_t budget_bytes, used_bytes, peak_used_bytes, reference_bytes;
    int workers, busy_workers, peak_busy_workers, queued;
    uint64_t admitted, workers_made, workers_released;
} shouji_server_stats;

shouji_status shouji_server_create(size_t max_request_pairs, uint32_t max_m,
                                   uint64_t max_stride, int e_min, int e_max,
                                   int with_n, size_t memory_budget,
                                   int max_slots, const char *tune_cache,
                                   shouji_server **out);

shouji_status shouji_server_info(shouji_server *server, int *slots,
                                 uint64_t *bytes_per_slot);

shouji_status shouji_server_stats_read(shouji_server *server, shouji_server_stats *out);

shouji_status shouji_server_add_reference(shouji_server *server, const uint8_t *text,
                                          uint64_t bytes, uint32_t *ref_id);

shouji_status shouji_server_submit_request(shouji_server *server,
                                           const shouji_server_request *request,
                                           uint64_t *request_id);

shouji_status shouji_server_submit(shouji_server *server, const uint8_t *reads,
                                   const uint8_t *refs, uint64_t stride,
                                   const uint16_t *lens,
                                   const uint8_t *E_per_pair, size_t n_pairs,
                                   uint32_t *accept, uint8_t *count,
                                   uint64_t *request_id);

shouji_status shouji_server_wait(shouji_server *server, uint64_t request_id,
                                 double timeout_s, double *latency_s);

shouji_status shouji_server_wait_timed(shouji_server *server, uint64_t request_id,
                                       double timeout_s, double *times);

void shouji_server_destroy(shouji_server *server);

#ifdef __cplusplus
}
#endif

#endif /* SHOUJI_H */
