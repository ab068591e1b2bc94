/*
 * Shouji CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct restatement of the Shouji pre-alignment
 * filter (Alser et al., "Shouji: a fast and efficient pre-alignment filter for
 * sequence alignment", arXiv 1809.07858), one pair at a time, on unpacked
 * ASCII bytes, with one plain loop per definition.  It exists to check the
 * CUDA path; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or layout with the CUDA
 * library, and it includes nothing from it.
 *
 * Notation follows the paper: P is the pattern (the read), T is the text (the
 * reference segment), both of length m; E is the edit distance threshold.
 * Indices are 0-based here (the paper is 1-based).
 *
 * Readings taken where the paper is silent, ambiguous or garbled (each one is
 * listed, with its evidence, in the design notes of the repository):
 *   R1  Orientation.  Rows of the neighborhood map index P, columns index T
 *       (Eq. 1).  Diagonal d holds, at column c, the comparison of P[c-d]
 *       with T[c]; d > 0 are the "upper" diagonals (P shifted right, Sec. 2.3)
 *       and d < 0 the "lower" ones, as printed in Fig. 6.
 *   R2  Window alignment.  Every 4-bit diagonal segment of search window c
 *       covers the same four columns c..c+3 (Sec. 2.2.2: "a search window of
 *       4 columns"; Sec. 2.3: every diagonal is a shifted copy of P compared
 *       with T at the same positions).
 *   R3  Cells outside the band (P index c-d outside [0,m)) are mismatches (1).
 *   R4  There are m windows (Sec. 2.2.2); columns c >= m read as 1 and are
 *       never written.
 *   R5  Per window the selection runs over all 2E+1 segments and restarts
 *       for every window (Sec. 2.2.2 Step 1), in the order lower_1, upper_1,
 *       lower_2, upper_2, ..., lower_E, upper_E: a segment replaces the
 *       current choice when it has more zeros, or the same number of zeros
 *       while it starts with a zero and the current choice does not ("the
 *       first one that has a leading zero").  The main diagonal is examined
 *       last and replaces the choice only with strictly more zeros
 *       (Algorithm 1, step 2).  With E = 0 the choice is the main segment.
 *   R6  The Shouji bit-vector takes the chosen segment only when the segment
 *       has strictly more zeros than the four bits it would overwrite
 *       (Algorithm 1, step 2).
 *   R7  Accept iff the number of ones in the Shouji bit-vector is at most E,
 *       i.e. CZ(Shouji) >= m - E (Sec. 2.2.3, Algorithm 1, step 3).
 *   R8  The base 'N' matches nothing, not even another 'N' (the paper is
 *       silent on ambiguous bases).
 *   R10 Local / glocal counting drops the runs of ones at the ends of the
 *       Shouji bit-vector; a vector with no zero counts m.  A pattern
 *       shorter than the text reads as out of the band past its end.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ---------------------------------------------------------------------- */
/* Step 1: the neighborhood map (Sec. 2.2.1, Eq. 1).                       */
/* map[(d + E) * m + c] = N entry of diagonal d at column c, d in [-E, E]. */
/* ---------------------------------------------------------------------- */
static int is_unknown_base(char x) { return x == 'N'; }

static void build_map(const char *P, int mp, const char *T, int m, int E,
                      uint8_t *map)
{
    for (int d = -E; d <= E; ++d) {
        for (int c = 0; c < m; ++c) {
            int i = c - d;               /* index into P (row of N) */
            uint8_t cell;
            if (i < 0 || i >= mp)
                cell = 1;                /* R3: outside the band */
            else if (is_unknown_base(P[i]) || is_unknown_base(T[c]))
                cell = 1;                /* R8 */
            else
                cell = (P[i] == T[c]) ? 0 : 1;   /* Eq. 1 */
            map[(size_t)(d + E) * m + c] = cell;
        }
    }
}

void oracle_neighborhood_map(const char *P, const char *T, int m, int E,
                             uint8_t *map)
{
    build_map(P, m, T, m, E, map);
}

/* Algorithm 2: CZ counts the zeros of a bit-vector. */
static int CZ(const uint8_t *bits, int len)
{
    int count = 0;
    for (int k = 0; k < len; ++k)
        if (bits[k] == 0)
            count = count + 1;
    return count;
}

/* The 4-bit segment of diagonal d in the window that starts at column c
 * (R2, R4: columns past the end read as 1). */
static void segment(const uint8_t *map, int m, int E, int d, int c,
                    uint8_t seg[4])
{
    for (int k = 0; k < 4; ++k)
        seg[k] = (c + k < m) ? map[(size_t)(d + E) * m + c + k] : 1;
}

/* Steps 1 and 2 for a pattern P of length mp against a text T of length m
 * (mp = m in the global mode of the paper; a shorter P reads as out of the
 * band past its end, as the dashes of Fig. 6(c)).  Fills shouji[0..m). */
static int shouji_vector(const char *P, int mp, const char *T, int m, int E,
                         uint8_t *shouji)
{
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    if (!map)
        return -1;

    /* Step 1 */
    build_map(P, mp, T, m, E, map);

    /* Step 2: the Shouji bit-vector starts as all ones. */
    for (int c = 0; c < m; ++c)
        shouji[c] = 1;

    for (int c = 0; c < m; ++c) {            /* m search windows (R4) */
        uint8_t Z[4], cand[4], cur[4];

        /* Sec. 2.2.2 Step 1: the segment with the most zeros (R5). */
        if (E == 0) {
            segment(map, m, E, 0, c, Z);
        } else {
            segment(map, m, E, -1, c, Z);    /* lower_1 is examined first */
            for (int j = 1; j <= E; ++j) {
                for (int side = 0; side < 2; ++side) {
                    int d = (side == 0) ? -j : +j;   /* lower_j, then upper_j */
                    if (d == -1)
                        continue;                    /* already the choice */
                    segment(map, m, E, d, c, cand);
                    int zc = CZ(cand, 4), zz = CZ(Z, 4);
                    if (zc > zz || (zc == zz && Z[0] == 1 && cand[0] == 0))
                        memcpy(Z, cand, 4);
                }
            }
            segment(map, m, E, 0, c, cand);  /* main diagonal, strict */
            if (CZ(cand, 4) > CZ(Z, 4))
                memcpy(Z, cand, 4);
        }

        /* Sec. 2.2.2 Step 2: keep Z if it holds more zeros (R6). */
        for (int k = 0; k < 4; ++k)
            cur[k] = (c + k < m) ? shouji[c + k] : 1;
        if (CZ(Z, 4) > CZ(cur, 4))
            for (int k = 0; k < 4; ++k)
                if (c + k < m)
                    shouji[c + k] = Z[k];
    }

    free(map);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Steps 1-3 for one pair.  Writes the Shouji bit-vector (m bytes, 0/1) to */
/* S when S is not NULL and returns the number of ones in it (the edit     */
/* estimate); the pair is accepted iff the return value is <= E.           */
/* Returns -1 on an allocation failure or a bad argument.                  */
/* ---------------------------------------------------------------------- */
int oracle_shouji(const char *P, const char *T, int m, int E, uint8_t *S)
{
    if (m <= 0 || E < 0)
        return -1;
    uint8_t *shouji = (uint8_t *)malloc((size_t)m);
    if (!shouji || shouji_vector(P, m, T, m, E, shouji) != 0) {
        free(shouji);
        return -1;
    }
    /* Step 3 (Sec. 2.2.3): count the ones. */
    int ones = m - CZ(shouji, m);
    if (S)
        memcpy(S, shouji, (size_t)m);
    free(shouji);
    return ones;
}

/* ---------------------------------------------------------------------- */
/* Local and semi-global ("glocal") counting (Sec. 2.2.3; Supplementary    */
/* Sec. 8, Fig. 6(c)): the ones of the Shouji bit-vector that lie in the   */
/* run at one or both of its ends are not counted.                         */
/*   mode 0 global: every one;                                             */
/*   mode 1 local: not the leading nor the trailing run of ones;           */
/*   mode 2 glocal: not the leading run; mode 3 glocal: not the trailing.  */
/* Reading R10: a vector without any zero has no end runs to drop (all of  */
/* it is mismatch) and counts m.                                           */
/* ---------------------------------------------------------------------- */
int oracle_count_mode(const uint8_t *S, int m, int mode)
{
    int first = -1, last = -1;
    for (int c = 0; c < m; ++c) {
        if (S[c] == 0) {
            if (first < 0)
                first = c;
            last = c;
        }
    }
    if (first < 0)
        return m;
    int lo = (mode == 1 || mode == 2) ? first : 0;
    int hi = (mode == 1 || mode == 3) ? last : m - 1;
    int ones = 0;
    for (int c = lo; c <= hi; ++c)
        if (S[c] == 1)
            ones = ones + 1;
    return ones;
}

/* The filter for a pattern P of length mp <= m against a text T of length
 * m, with the count mode above; S (m bytes) may be NULL.  Returns the
 * count, or -1 on a bad argument or an allocation failure. */
int oracle_shouji_mode(const char *P, int mp, const char *T, int m, int E,
                       int mode, uint8_t *S)
{
    if (m <= 0 || mp < 0 || mp > m || E < 0 || mode < 0 || mode > 3)
        return -1;
    uint8_t *shouji = (uint8_t *)malloc((size_t)m);
    if (!shouji || shouji_vector(P, mp, T, m, E, shouji) != 0) {
        free(shouji);
        return -1;
    }
    int count = oracle_count_mode(shouji, m, mode);
    if (S)
        memcpy(S, shouji, (size_t)m);
    free(shouji);
    return count;
}

/* ---------------------------------------------------------------------- */
/* Global edit distance (Levenshtein; unit-cost substitutions, insertions  */
/* and deletions, end to end), by the full dynamic-programming table.  It  */
/* is the ground truth the paper takes from Edlib in its global mode when  */
/* it counts false accepts and false rejects (Sec. 3.2).                   */
/* ---------------------------------------------------------------------- */
int oracle_edit_distance(const char *a, int la, const char *b, int lb)
{
    int *prev = (int *)malloc(sizeof(int) * (size_t)(lb + 1));
    int *next = (int *)malloc(sizeof(int) * (size_t)(lb + 1));
    if (!prev || !next) {
        free(prev);
        free(next);
        return -1;
    }
    for (int j = 0; j <= lb; ++j)
        prev[j] = j;
    for (int i = 1; i <= la; ++i) {
        next[0] = i;
        for (int j = 1; j <= lb; ++j) {
            int sub = prev[j - 1] + (a[i - 1] == b[j - 1] ? 0 : 1);
            int del = prev[j] + 1;
            int ins = next[j - 1] + 1;
            int best = sub < del ? sub : del;
            next[j] = best < ins ? best : ins;
        }
        int *t = prev;
        prev = next;
        next = t;
    }
    int d = prev[lb];
    free(prev);
    free(next);
    return d;
}

/* ---------------------------------------------------------------------- */
/* Batch driver: pairs (reads + i*stride, refs + i*stride), m bytes each.  */
/* E_per_pair overrides E when not NULL.  accept[i] = 1/0, count[i] = the  */
/* ones in the Shouji bit-vector (capped at 255 only by the type).  The    */
/* pairs are split into contiguous ranges, one per thread.  Returns 0, or  */
/* -1 on a failure.                                                        */
/* ---------------------------------------------------------------------- */
typedef struct {
    const char *reads, *refs;
    size_t stride;
    int m, E;
    const uint8_t *E_per_pair;
    uint8_t *accept, *count;
    size_t lo, hi;
    int failed;
    int magnet;  /* 0: Shouji, 1: MAGNET (global count) */
} batch_job;

int oracle_magnet_mode(const char *P, int mp, const char *T, int m, int E, int mode,
                       uint8_t *V);

static void *batch_worker(void *arg)
{
    batch_job *job = (batch_job *)arg;
    for (size_t i = job->lo; i < job->hi; ++i) {
        int E = job->E_per_pair ? job->E_per_pair[i] : job->E;
        const char *P = job->reads + i * job->stride, *T = job->refs + i * job->stride;
        int ones = job->magnet ? oracle_magnet_mode(P, job->m, T, job->m, E, 0, NULL)
                               : oracle_shouji(P, T, job->m, E, NULL);
        if (ones < 0) {
            job->failed = 1;
            return NULL;
        }
        if (job->accept)
            job->accept[i] = (uint8_t)(ones <= E);
        if (job->count)
            job->count[i] = (uint8_t)ones;
    }
    return NULL;
}

static int run_batch(const char *reads, const char *refs, size_t stride, int m, size_t n,
                     int E, const uint8_t *E_per_pair, uint8_t *accept, uint8_t *count,
                     int threads, int magnet)
{
    if (threads < 1)
        threads = 1;
    if ((size_t)threads > n && n > 0)
        threads = (int)n;
    batch_job *jobs = (batch_job *)calloc((size_t)threads, sizeof(batch_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !tids) {
        free(jobs);
        free(tids);
        return -1;
    }
    size_t per = n / (size_t)threads, extra = n % (size_t)threads, at = 0;
    for (int t = 0; t < threads; ++t) {
        size_t len = per + ((size_t)t < extra ? 1 : 0);
        jobs[t] = (batch_job){reads, refs, stride, m, E, E_per_pair,
                              accept, count, at, at + len, 0, magnet};
        at += len;
    }
    int failed = 0;
    if (threads == 1) {
        batch_worker(&jobs[0]);
    } else {
        for (int t = 0; t < threads; ++t)
            if (pthread_create(&tids[t], NULL, batch_worker, &jobs[t]) != 0)
                jobs[t].failed = 2;
        for (int t = 0; t < threads; ++t)
            if (jobs[t].failed != 2)
                pthread_join(tids[t], NULL);
    }
    for (int t = 0; t < threads; ++t)
        failed |= jobs[t].failed;
    free(jobs);
    free(tids);
    return failed ? -1 : 0;
}

int oracle_shouji_batch(const char *reads, const char *refs, size_t stride,
                        int m, size_t n, int E, const uint8_t *E_per_pair,
                        uint8_t *accept, uint8_t *count, int threads)
{
    return run_batch(reads, refs, stride, m, n, E, E_per_pair, accept, count, threads, 0);
}

/* MAGNET over a batch of equal-length pairs (global count), as above. */
int oracle_magnet_batch(const char *reads, const char *refs, size_t stride,
                        int m, size_t n, int E, const uint8_t *E_per_pair,
                        uint8_t *accept, uint8_t *count, int threads)
{
    return run_batch(reads, refs, stride, m, n, E, E_per_pair, accept, count, threads, 1);
}

/* ====================================================================== */
/* MAGNET (Supplementary Sec. 7, Algorithms 3 and 4): the paper's second  */
/* filter on the same neighborhood map.  Readings (listed with evidence   */
/* in the design notes):                                                  */
/*   M1  As in Algorithm 1, the printed extraction loop overwrites its     */
/*       choice for every j; the prose selects the longest of all 2E+1     */
/*       diagonals' runs, so the choice is a running best.                 */
/*   M2  Diagonal j's pair: the lower run wins only when strictly longer   */
/*       (Algorithm 4 prefers the upper on ties); a pair's winner replaces */
/*       the best so far only when strictly longer (the first j wins ties);*/
/*       the main diagonal replaces it only when strictly longer.          */
/*   M3  CCZ returns the longest run of consecutive zeros of a diagonal    */
/*       inside columns [SI, EI], the leftmost of equally long runs.       */
/*   M4  The extracted run's columns become zeros of the MAGNET vector;    */
/*       the columns just before and after it (the encapsulation bits)     */
/*       stay ones; subproblems cover [e+2, EI] (first) and [SI, s-2].     */
/*   M5  The counter `calls` counts extractions in the order they happen   */
/*       (a call that extracts nothing gives its number back); at most     */
/*       E+1 extractions.  A range without any zero extracts nothing.      */
/*   M6  Only the first extraction checks the length bound: a longest run  */
/*       shorter than ceil((m-E)/(E+1)) rejects the pair at once (the      */
/*       MAGNET vector stays all ones).                                    */
/* ====================================================================== */
typedef struct {
    const uint8_t *map;
    int m, E;
    uint8_t *vec;
    int rejected;
} magnet_state;

/* CCZ: longest run of zeros of diagonal d inside [SI, EI] (M3). */
static int CCZ(const magnet_state *st, int d, int SI, int EI, int *s_out, int *e_out)
{
    int best = 0, bs = -1, run = 0;
    for (int c = SI; c <= EI; ++c) {
        if (st->map[(size_t)(d + st->E) * st->m + c] == 0) {
            ++run;
            if (run > best) {
                best = run;
                bs = c - run + 1;
            }
        } else {
            run = 0;
        }
    }
    *s_out = bs;
    *e_out = bs + best - 1;
    return best;
}

static int EXEN(magnet_state *st, int SI, int EI, int calls)
{
    const int E = st->E;
    if (!(SI <= EI && calls <= E + 1))
        return calls - 1;
    /* Extraction (M1, M2) */
    int len = 0, s = -1, e = -2;
    for (int j = 1; j <= E; ++j) {
        int s1, e1, s2, e2;
        int X = CCZ(st, -j, SI, EI, &s1, &e1);   /* lower diagonal j */
        int Y = CCZ(st, +j, SI, EI, &s2, &e2);   /* upper diagonal j */
        int L = X > Y ? X : Y;
        int ls = X > Y ? s1 : s2, le = X > Y ? e1 : e2;
        if (L > len) {
            len = L;
            s = ls;
            e = le;
        }
    }
    {
        int s1, e1;
        int X = CCZ(st, 0, SI, EI, &s1, &e1);   /* main diagonal */
        if (X > len) {
            len = X;
            s = s1;
            e = e1;
        }
    }
    if (len == 0)
        return calls - 1;                         /* nothing to extract (M5) */
    /* Early termination, first call only (M6) */
    if (calls == 1 && len < (st->m - E + E) / (E + 1)) {  /* ceil((m-E)/(E+1)) */
        st->rejected = 1;
        return 0;
    }
    for (int c = s; c <= e; ++c)
        st->vec[c] = 0;                           /* M4 */
    calls = EXEN(st, e + 2, EI, calls + 1);       /* right subproblem */
    calls = EXEN(st, SI, s - 2, calls + 1);       /* left subproblem */
    return calls;
}

/* MAGNET for a pattern P of length mp <= m against a text T of length m,
 * with the count modes of oracle_count_mode.  Writes the MAGNET vector to V
 * (m bytes) when not NULL; returns the count, or -1. */
int oracle_magnet_mode(const char *P, int mp, const char *T, int m, int E, int mode,
                       uint8_t *V)
{
    if (m <= 0 || mp < 0 || mp > m || E < 0 || mode < 0 || mode > 3)
        return -1;
    uint8_t *map = (uint8_t *)malloc((size_t)(2 * E + 1) * m);
    uint8_t *vec = (uint8_t *)malloc((size_t)m);
    if (!map || !vec) {
        free(map);
        free(vec);
        return -1;
    }
    build_map(P, mp, T, m, E, map);
    for (int c = 0; c < m; ++c)
        vec[c] = 1;
    magnet_state st = {map, m, E, vec, 0};
    EXEN(&st, 0, m - 1, 1);
    if (st.rejected)
        for (int c = 0; c < m; ++c)
            vec[c] = 1;
    int count = oracle_count_mode(vec, m, mode);
    if (V)
        memcpy(V, vec, (size_t)m);
    free(map);
    free(vec);
    return count;
}
