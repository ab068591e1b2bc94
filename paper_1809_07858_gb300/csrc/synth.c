/*
 * Seeded synthetic read / reference-segment pairs shaped like the workloads
 * of the Shouji paper (arXiv 1809.07858, Sec. 3.1: pairs of equal length
 * 100/150/250 bp, edit thresholds up to 10% of the length, a mix of
 * low-edit and high-edit pairs).  The paper's real datasets are not
 * available, so these pairs stand in for them.
 *
 * This file holds no part of the filter's arithmetic.  It is the one input
 * source shared by the CUDA path's tests/benchmark and by the CPU oracle's
 * tests, and it depends on neither.
 *
 * Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used counter-style: pair i
 * owns the stream seeded by (seed, i), so any sub-range of pairs can be
 * regenerated alone, on any number of threads, with identical bytes.
 *
 * Recipe for pair i (read = pattern P, reference segment = text T):
 *   1. read: m bases drawn uniformly from {A,C,G,T};
 *   2. the pair is "far" with probability far_fraction, else "near";
 *      k is uniform in [near_kmin, near_kmax] or [far_kmin, far_kmax];
 *   3. ref = read with k edits applied one after another; each edit is a
 *      substitution, an insertion or a deletion with probability 1/3 each,
 *      at a position uniform over the current sequence (insertion: over the
 *      len+1 gaps); a substitution draws one of the 3 other bases, an
 *      inserted base is uniform; a deletion or substitution on an empty
 *      sequence does nothing;
 *   4. ref is trimmed to m, or padded with uniform bases up to m;
 *   5. with n_rate > 0, every base of read and ref independently becomes 'N'
 *      with probability n_rate.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef struct {
    uint64_t state;
} sm64_t;

static inline uint64_t sm64_next(sm64_t *g)
{
    uint64_t z = (g->state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform integer in [0, n), n >= 1 (multiply-shift on the high 32 bits). */
static inline uint32_t sm64_below(sm64_t *g, uint32_t n)
{
    return (uint32_t)(((sm64_next(g) >> 32) * (uint64_t)n) >> 32);
}

/* Uniform double in [0, 1) from the high 53 bits. */
static inline double sm64_unit(sm64_t *g)
{
    return (double)(sm64_next(g) >> 11) * (1.0 / 9007199254740992.0);
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static inline int base_code(char b)
{
    switch (b) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    default: return 3;
    }
}

typedef struct {
    uint64_t seed;
    uint64_t first;
    uint32_t m;
    uint64_t stride;
    uint32_t near_kmin, near_kmax, far_kmin, far_kmax;
    double far_fraction, n_rate;
    const uint16_t *lengths; /* optional per-pair length (<= m) */
    uint8_t *reads, *refs;
    uint8_t *kind_out;       /* optional: 0 near / 1 far */
    uint8_t *k_out;          /* optional: edits applied (capped at 255) */
    uint64_t lo, hi;
} synth_job;

static void make_pair(const synth_job *J, uint64_t i, char *work)
{
    uint64_t gi = J->first + i;
    sm64_t g = {J->seed * 0xD1B54A32D192ED03ull + (gi + 1) * 0x9E3779B97F4A7C15ull};
    sm64_next(&g);
    uint32_t m = J->lengths ? J->lengths[i] : J->m;
    char *read = (char *)J->reads + i * J->stride;
    char *ref = (char *)J->refs + i * J->stride;

    for (uint32_t c = 0; c < m; c += 32) {
        uint64_t bits = sm64_next(&g);
        for (uint32_t k = 0; k < 32 && c + k < m; ++k)
            read[c + k] = BASES[(bits >> (2 * k)) & 3];
    }

    int far = J->far_fraction > 0.0 && sm64_unit(&g) < J->far_fraction;
    uint32_t klo = far ? J->far_kmin : J->near_kmin;
    uint32_t khi = far ? J->far_kmax : J->near_kmax;
    uint32_t k = klo + sm64_below(&g, khi - klo + 1);

    uint32_t len = m;
    memcpy(work, read, m);
    for (uint32_t e = 0; e < k; ++e) {
        uint32_t type = sm64_below(&g, 3);
        if (type == 0) {                 /* substitution */
            if (len == 0)
                continue;
            uint32_t pos = sm64_below(&g, len);
            int old = base_code(work[pos]);
            work[pos] = BASES[(old + 1 + (int)sm64_below(&g, 3)) & 3];
        } else if (type == 1) {          /* insertion */
            uint32_t pos = sm64_below(&g, len + 1);
            memmove(work + pos + 1, work + pos, len - pos);
            work[pos] = BASES[sm64_below(&g, 4)];
            ++len;
        } else {                         /* deletion */
            if (len == 0)
                continue;
            uint32_t pos = sm64_below(&g, len);
            memmove(work + pos, work + pos + 1, len - pos - 1);
            --len;
        }
    }
    if (len > m)
        len = m;
    while (len < m)
        work[len++] = BASES[sm64_below(&g, 4)];
    memcpy(ref, work, m);

    if (J->n_rate > 0.0) {
        for (uint32_t c = 0; c < m; ++c)
            if (sm64_unit(&g) < J->n_rate)
                read[c] = 'N';
        for (uint32_t c = 0; c < m; ++c)
            if (sm64_unit(&g) < J->n_rate)
                ref[c] = 'N';
    }
    if (J->kind_out)
        J->kind_out[i] = (uint8_t)far;
    if (J->k_out)
        J->k_out[i] = (uint8_t)(k > 255 ? 255 : k);
}

static void *synth_worker(void *arg)
{
    synth_job *J = (synth_job *)arg;
    uint32_t kmax = J->near_kmax > J->far_kmax ? J->near_kmax : J->far_kmax;
    char *work = (char *)malloc((size_t)J->m + kmax + 1);
    if (!work)
        return (void *)1;
    for (uint64_t i = J->lo; i < J->hi; ++i)
        make_pair(J, i, work);
    free(work);
    return NULL;
}

/*
 * Generate pairs first .. first+n-1 into reads/refs (row i at i*stride,
 * m bytes, or lengths[i] bytes when lengths is not NULL; bytes past a row's
 * length are left untouched).  Returns 0, or -1 on a bad argument or an
 * allocation failure.
 */
int synth_pairs(uint64_t seed, uint64_t first, uint64_t n, uint32_t m,
                uint64_t stride, uint32_t near_kmin, uint32_t near_kmax,
                uint32_t far_kmin, uint32_t far_kmax, double far_fraction,
                double n_rate, const uint16_t *lengths, uint8_t *reads,
                uint8_t *refs, uint8_t *kind_out, uint8_t *k_out, int threads)
{
    if (stride < m || near_kmin > near_kmax ||
        (far_fraction > 0.0 && far_kmin > far_kmax) || !reads || !refs)
        return -1;
    if (threads < 1)
        threads = 1;
    if ((uint64_t)threads > n)
        threads = n ? (int)n : 1;
    synth_job *jobs = (synth_job *)calloc((size_t)threads, sizeof(synth_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return -1;
    }
    uint64_t per = n / (uint64_t)threads, extra = n % (uint64_t)threads, at = 0;
    for (int t = 0; t < threads; ++t) {
        uint64_t len = per + ((uint64_t)t < extra ? 1 : 0);
        jobs[t] = (synth_job){seed, first, m, stride, near_kmin, near_kmax,
                              far_kmin, far_kmax, far_fraction, n_rate,
                              lengths, reads, refs, kind_out, k_out, at, at + len};
        at += len;
    }
    int failed = 0;
    if (threads == 1) {
        failed = synth_worker(&jobs[0]) != NULL;
    } else {
        int *started = (int *)calloc((size_t)threads, sizeof(int));
        for (int t = 0; t < threads; ++t)
            started[t] = pthread_create(&tids[t], NULL, synth_worker, &jobs[t]) == 0;
        for (int t = 0; t < threads; ++t) {
            if (!started[t]) {
                failed = 1;
                continue;
            }
            void *rv = NULL;
            pthread_join(tids[t], &rv);
            failed |= rv != NULL;
        }
        free(started);
    }
    free(jobs);
    free(tids);
    return failed ? -1 : 0;
}

/*
 * Per-pair lengths and thresholds for mixed batches: length drawn from
 * `choices` (n_choices values) with cumulative weights `cum` (last = 1.0),
 * E uniform in [e_min, e_max].  Stream (seed, first + i) as above, but on a
 * separate seed lane so it does not correlate with synth_pairs.
 */
int synth_mixed_shape(uint64_t seed, uint64_t first, uint64_t n,
                      const uint16_t *choices, const double *cum, int n_choices,
                      uint32_t e_min, uint32_t e_max, uint16_t *lengths,
                      uint8_t *E_out)
{
    if (n_choices < 1 || e_min > e_max)
        return -1;
    for (uint64_t i = 0; i < n; ++i) {
        sm64_t g = {(seed ^ 0x5DEECE66Dull) * 0xD1B54A32D192ED03ull +
                    (first + i + 1) * 0x9E3779B97F4A7C15ull};
        sm64_next(&g);
        double u = sm64_unit(&g);
        int j = 0;
        while (j < n_choices - 1 && u >= cum[j])
            ++j;
        if (lengths)
            lengths[i] = choices[j];
        if (E_out)
            E_out[i] = (uint8_t)(e_min + sm64_below(&g, e_max - e_min + 1));
    }
    return 0;
}
