/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for exact matching of
 * DNA queries by binary search over a suffix array.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or helper with the CUDA
 * library and does not include anything from it.
 *
 * Text model (Section III): a reference S over Sigma = {a,c,g,t}, n = |S|,
 * suffixes S_i = S(i,n).  The oracle stores one byte per base, folded to the
 * upper-case letters 'A' < 'C' < 'G' < 'T', whose byte order is the
 * lexicographic order of Sigma.  Positions are 0-based as in Table I.
 *
 * Every routine states the passage it follows.  Readings taken where the paper
 * is silent or garbled:
 *   R1  Alg. 1's bound tests are read as the standard lower/upper bound:
 *       LB is the first rank with P <= m-prefix(suffix), and RB + 1 the
 *       first rank with P < m-prefix(suffix).
 *   R2  The search covers every rank: Alg. 1's boundaries -1 and n are the
 *       exclusive ends of the range [0, n).
 *   R3  No terminator is printed; Table I orders a proper prefix before any
 *       longer suffix that starts with it, so a suffix that ends before the
 *       query does compares smaller than the query.
 *   R4  The closed interval [LB,RB] of Section IV is reported half-open:
 *       lo = LB, hi = RB + 1, count = hi - lo.
 *   R5  A miss gives lo = hi = the insertion point, count = 0.
 *   R6  m = 0 matches every suffix: [0, n).
 *   R7  Located positions are reported in suffix-array order.
 *
 * Parity status: every function here is pinned by tests (Tables I-III, the
 * Section IV examples, brute force on exhaustive tiny inputs, closed forms
 * for probe counts); nothing is unpinned.
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* Alphabet (Section III: Sigma = {a,c,g,t})                           */
/* ------------------------------------------------------------------ */

/* Fold a/c/g/t to upper case.  Returns 0, or -1 and the index of the first
 * byte outside {A,C,G,T,a,c,g,t} in *bad. */
int oracle_normalize(const uint8_t *in, int64_t n, uint8_t *out, int64_t *bad)
{
    for (int64_t i = 0; i < n; i++) {
        uint8_t c = in[i];
        if (c >= 'a' && c <= 'z')
            c = (uint8_t)(c - 'a' + 'A');
        if (c != 'A' && c != 'C' && c != 'G' && c != 'T') {
            if (bad)
                *bad = i;
            return -1;
        }
        out[i] = c;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Suffix order (Section III, Fig. 3, Table I)                         */
/* ------------------------------------------------------------------ */

/* Lexicographic comparison of suffixes S_i and S_j of T[0..n); a suffix
 * that is a proper prefix of the other is the smaller one (reading R3). */
static int suffix_cmp(const uint8_t *T, int64_t n, int64_t i, int64_t j)
{
    if (i == j)
        return 0;
    int64_t li = n - i, lj = n - j;
    int64_t k = li < lj ? li : lj;
    for (int64_t t = 0; t < k; t++) {
        if (T[i + t] != T[j + t])
            return T[i + t] < T[j + t] ? -1 : 1;
    }
    return li < lj ? -1 : 1;
}

struct sort_ctx {
    const uint8_t *T;
    int64_t n;
};

static int qsort_suffix_cmp(const void *a, const void *b, void *arg)
{
    const struct sort_ctx *c = (const struct sort_ctx *)arg;
    return suffix_cmp(c->T, c->n, *(const int64_t *)a, *(const int64_t *)b);
}

/* The straightforward construction of Section III: place every suffix start
 * in an array and sort it with a comparison sort. */
void oracle_sa_naive(const uint8_t *T, int64_t n, int64_t *sa)
{
    for (int64_t i = 0; i < n; i++)
        sa[i] = i;
    struct sort_ctx c = {T, n};
    qsort_r(sa, (size_t)n, sizeof(int64_t), qsort_suffix_cmp, &c);
}

/* Inverse suffix array, 1-based: rank1[SA[k]] = k + 1 (Table III). */
void oracle_ranks(const int64_t *sa, int64_t n, int64_t *rank1)
{
    for (int64_t k = 0; k < n; k++)
        rank1[sa[k]] = k + 1;
}

/* Checks that sa is THE suffix array of T: a permutation of [0,n) whose
 * adjacent suffixes are strictly increasing.  The suffixes of a string are
 * pairwise distinct, so a sorted permutation is unique and this check proves
 * equality with any correct construction.  Returns 0 if valid; 1 if a value
 * is out of range, 2 if a value repeats, 3 if an adjacent pair is out of
 * order; *where receives the offending index. */
static int verify_range(const uint8_t *T, int64_t n, const int64_t *sa,
                        int64_t a, int64_t b, int64_t *where)
{
    for (int64_t k = a; k < b; k++) {
        if (suffix_cmp(T, n, sa[k], sa[k + 1]) >= 0) {
            *where = k;
            return 3;
        }
    }
    return 0;
}

struct verify_job {
    const uint8_t *T;
    int64_t n;
    const int64_t *sa;
    int64_t a, b, where;
    int rc;
};

static void *verify_worker(void *p)
{
    struct verify_job *j = (struct verify_job *)p;
    j->rc = verify_range(j->T, j->n, j->sa, j->a, j->b, &j->where);
    return NULL;
}

struct perm_job {
    const int64_t *sa;
    int64_t n, a, b, where;
    uint8_t *seen;
    int rc;
};

/* Marks the values of sa[a..b) in seen; a value out of range, or one already
 * marked (by this thread or another), is reported. */
static void *perm_worker(void *p)
{
    struct perm_job *j = (struct perm_job *)p;
    for (int64_t k = j->a; k < j->b; k++) {
        int64_t v = j->sa[k];
        if (v < 0 || v >= j->n) {
            j->rc = 1;
            j->where = k;
            return NULL;
        }
        if (__atomic_exchange_n(&j->seen[v], (uint8_t)1, __ATOMIC_RELAXED)) {
            j->rc = 2;
            j->where = k;
            return NULL;
        }
    }
    return NULL;
}

int oracle_verify_sa(const uint8_t *T, int64_t n, const int64_t *sa,
                     int nthreads, int64_t *where)
{
    int64_t w = -1;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > n)
        nthreads = n > 0 ? (int)n : 1;
    /* Permutation of [0, n): every value in range and none repeated. */
    uint8_t *seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    struct perm_job *pj = (struct perm_job *)calloc((size_t)nthreads, sizeof *pj);
    pthread_t *pth = (pthread_t *)calloc((size_t)nthreads, sizeof *pth);
    if (!seen || !pj || !pth) {
        free(seen);
        free(pj);
        free(pth);
        return -1;
    }
    for (int t = 0; t < nthreads; t++) {
        pj[t].sa = sa;
        pj[t].n = n;
        pj[t].a = n * t / nthreads;
        pj[t].b = n * (t + 1) / nthreads;
        pj[t].seen = seen;
        pthread_create(&pth[t], NULL, perm_worker, &pj[t]);
    }
    int prc = 0;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(pth[t], NULL);
        if (pj[t].rc && (!prc || pj[t].rc < prc)) {
            prc = pj[t].rc;
            w = pj[t].where;
        }
    }
    free(seen);
    free(pj);
    free(pth);
    if (prc) {
        if (where)
            *where = w;
        return prc;
    }
    if (n < 2)
        return 0;
    int64_t pairs = n - 1;
    if (nthreads > pairs)
        nthreads = (int)pairs;
    struct verify_job *jobs = (struct verify_job *)calloc((size_t)nthreads, sizeof *jobs);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof *th);
    for (int t = 0; t < nthreads; t++) {
        jobs[t].T = T;
        jobs[t].n = n;
        jobs[t].sa = sa;
        jobs[t].a = pairs * t / nthreads;
        jobs[t].b = pairs * (t + 1) / nthreads;
        pthread_create(&th[t], NULL, verify_worker, &jobs[t]);
    }
    int rc = 0;
    for (int t = 0; t < nthreads; t++) {
        pthread_join(th[t], NULL);
        if (jobs[t].rc && !rc) {
            rc = jobs[t].rc;
            w = jobs[t].where;
        }
    }
    free(jobs);
    free(th);
    if (where)
        *where = w;
    return rc;
}

/* ------------------------------------------------------------------ */
/* Query against suffix (Section IV, the three cases)                  */
/* ------------------------------------------------------------------ */

/* Compares query P (length m) with the m-prefix of suffix S_p.
 * Returns -1 if P sorts before it (case 2 of Section IV), 0 if P is a
 * prefix of S_p (case 1), +1 if P sorts after it (case 3).  A suffix that
 * ends before P does sorts before P (reading R3).  *lcp receives the length
 * of the common prefix of P and S_p, capped at m. */
static int query_cmp(const uint8_t *T, int64_t n, int64_t p,
                     const uint8_t *P, int64_t m, int64_t *lcp)
{
    for (int64_t k = 0; k < m; k++) {
        if (p + k >= n) {
            if (lcp)
                *lcp = k;
            return 1;
        }
        if (T[p + k] != P[k]) {
            if (lcp)
                *lcp = k;
            return P[k] < T[p + k] ? -1 : 1;
        }
    }
    if (lcp)
        *lcp = m;
    return 0;
}

/* The interval of Section IV for one query, by two binary searches over the
 * suffix array -- the search Alg. 1 performs on the GPU, written here as the
 * textbook lower and upper bound over the half-open range of ranks [0, n)
 * (R2: every rank can be an answer).  lo is the first rank whose suffix's
 * m-prefix does not sort before P (R1, R3); hi is the first rank whose
 * suffix's m-prefix sorts after P.  Every rank in [lo, hi) has P as a prefix
 * (R4); a miss gives lo = hi (R5). */
void oracle_search(const uint8_t *T, int64_t n, const int64_t *sa,
                   const uint8_t *P, int64_t m, int64_t *lo, int64_t *hi)
{
    int64_t a = 0, b = n; /* the lower bound lies in [a, b] */
    while (a < b) {
        int64_t mid = a + (b - a) / 2;
        if (query_cmp(T, n, sa[mid], P, m, NULL) > 0) /* S_SA[mid] sorts before P */
            a = mid + 1;
        else
            b = mid;
    }
    *lo = a;
    b = n; /* the upper bound lies in [lo, n] */
    while (a < b) {
        int64_t mid = a + (b - a) / 2;
        if (query_cmp(T, n, sa[mid], P, m, NULL) >= 0) /* S_SA[mid] does not sort after P */
            a = mid + 1;
        else
            b = mid;
    }
    *hi = a;
}

/* The interval by its definition, without a suffix array: lo is the number
 * of suffixes whose m-prefix sorts before P, hi the number whose m-prefix
 * sorts before P or has P as prefix (Section IV: the suffixes with P as a
 * prefix form one contiguous range of the sorted order). */
void oracle_rank_count(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m,
                       int64_t *lo, int64_t *hi)
{
    int64_t less = 0, prefix = 0;
    for (int64_t i = 0; i < n; i++) {
        int c = query_cmp(T, n, i, P, m, NULL);
        if (c > 0)
            less++;
        else if (c == 0)
            prefix++;
    }
    *lo = less;
    *hi = less + prefix;
}

/* Every occurrence of P in T, overlapping ones included, by scanning each
 * text position.  Writes up to cap positions in increasing position order;
 * returns the total number of occurrences. */
int64_t oracle_bruteforce(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m,
                          int64_t *pos, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t i = 0; i + m <= n; i++) {
        if (memcmp(T + i, P, (size_t)m) == 0) {
            if (cnt < cap && pos)
                pos[cnt] = i;
            cnt++;
        }
    }
    return cnt;
}

/* Sorts a list of text positions into suffix order (R7: located positions
 * come out in suffix-array order). */
void oracle_sort_positions(const uint8_t *T, int64_t n, int64_t *pos, int64_t k)
{
    struct sort_ctx c = {T, n};
    qsort_r(pos, (size_t)k, sizeof(int64_t), qsort_suffix_cmp, &c);
}

/* ------------------------------------------------------------------ */
/* Batches over threads (the paper's CPU baseline runs queries in      */
/* parallel with OpenMP, Section V; plain pthreads here)              */
/* ------------------------------------------------------------------ */

struct batch_job {
    const uint8_t *T;
    int64_t n;
    const int64_t *sa;
    const uint8_t *Q;
    const int64_t *qoff;
    int64_t a, b;
    int64_t *lo, *hi;
    int mode; /* 0 = Alg. 1 search, 1 = definition count */
};

static void *batch_worker(void *p)
{
    struct batch_job *j = (struct batch_job *)p;
    for (int64_t q = j->a; q < j->b; q++) {
        const uint8_t *P = j->Q + j->qoff[q];
        int64_t m = j->qoff[q + 1] - j->qoff[q];
        if (j->mode == 0)
            oracle_search(j->T, j->n, j->sa, P, m, &j->lo[q], &j->hi[q]);
        else
            oracle_rank_count(j->T, j->n, P, m, &j->lo[q], &j->hi[q]);
    }
    return NULL;
}

static void run_batch(const uint8_t *T, int64_t n, const int64_t *sa,
                      const uint8_t *Q, const int64_t *qoff, int64_t nq,
                      int64_t *lo, int64_t *hi, int nthreads, int mode)
{
    if (nq <= 0)
        return;
    if (nthreads < 1)
        nthreads = 1;
    if (nthreads > nq)
        nthreads = (int)nq;
    struct batch_job *jobs = (struct batch_job *)calloc((size_t)nthreads, sizeof *jobs);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof *th);
    for (int t = 0; t < nthreads; t++) {
        struct batch_job j = {T, n, sa, Q, qoff, nq * t / nthreads,
                              nq * (t + 1) / nthreads, lo, hi, mode};
        jobs[t] = j;
        pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++)
        pthread_join(th[t], NULL);
    free(jobs);
    free(th);
}

/* Queries are concatenated in Q; query q is Q[qoff[q] .. qoff[q+1]). */
void oracle_search_batch(const uint8_t *T, int64_t n, const int64_t *sa,
                         const uint8_t *Q, const int64_t *qoff, int64_t nq,
                         int64_t *lo, int64_t *hi, int nthreads)
{
    run_batch(T, n, sa, Q, qoff, nq, lo, hi, nthreads, 0);
}

void oracle_rank_count_batch(const uint8_t *T, int64_t n,
                             const uint8_t *Q, const int64_t *qoff, int64_t nq,
                             int64_t *lo, int64_t *hi, int nthreads)
{
    run_batch(T, n, NULL, Q, qoff, nq, lo, hi, nthreads, 1);
}

/* Locate: the first min(count, cap) suffix-array entries of the interval,
 * in suffix-array order (R7). */
void oracle_locate(const int64_t *sa, int64_t lo, int64_t hi, int64_t cap, int64_t *out)
{
    int64_t c = hi - lo;
    if (c > cap)
        c = cap;
    for (int64_t k = 0; k < c; k++)
        out[k] = sa[lo + k];
}

/* ------------------------------------------------------------------ */
/* Byte model of one query's search (measurement, not a parity output) */
/* ------------------------------------------------------------------ */

/* Simulates a lockstep lower/upper-bound search over the boundaries
 * L = -1, R = n: while both bounds share (L,R) one probe serves both; when
 * the pivot's suffix has P as a prefix the searches split and each bound
 * continues alone.  Each compare starts at min(lcp(P,S_L), lcp(P,S_R)),
 * rounded down to a multiple of 64 bases, and reads 64-base chunks until the
 * comparison is decided.  Probes at depth >= d0 (the first probe has depth
 * 0) are counted in *probes and their chunks in *chunks.  Returns lo and hi
 * (which must equal the search results). */
static void model_probe(const uint8_t *T, int64_t n, const int64_t *sa,
                        const uint8_t *P, int64_t m, int64_t pivot,
                        int64_t lcpL, int64_t lcpR, int depth, int d0,
                        int *res, int64_t *lcp, int64_t *probes, int64_t *chunks)
{
    int64_t start = lcpL < lcpR ? lcpL : lcpR;
    start -= start % 64;
    int64_t l;
    int c = query_cmp(T, n, sa[pivot], P, m, &l);
    /* The compare looks at positions start .. last, where last is the
     * mismatch, the end of the suffix or the last base of P. */
    int64_t last = l < m - 1 ? l : m - 1;
    if (last < start)
        last = start;
    int64_t nch = last / 64 - start / 64 + 1;
    if (depth >= d0) {
        (*probes)++;
        (*chunks) += nch;
    }
    *res = c;
    *lcp = l;
}

void oracle_probe_model(const uint8_t *T, int64_t n, const int64_t *sa,
                        const uint8_t *P, int64_t m, int d0,
                        int64_t *probes, int64_t *chunks, int64_t *lo, int64_t *hi)
{
    *probes = 0;
    *chunks = 0;
    int64_t L = -1, R = n, lcpL = 0, lcpR = 0;
    int depth = 0;
    int c;
    int64_t l;
    /* Lockstep phase. */
    while (R > L + 1) {
        int64_t pivot = (L + R) >> 1;
        model_probe(T, n, sa, P, m, pivot, lcpL, lcpR, depth, d0, &c, &l, probes, chunks);
        depth++;
        if (c < 0) {
            R = pivot;
            lcpR = l;
        } else if (c > 0) {
            L = pivot;
            lcpL = l;
        } else {
            break;
        }
    }
    if (R <= L + 1) {
        *lo = R;
        *hi = R;
        return;
    }
    /* Split at the pivot whose suffix has P as a prefix. */
    int64_t split = (L + R) >> 1;
    int sdepth = depth;
    /* Lower bound in (L, split]. */
    int64_t a = L, b = split, la = lcpL, lb = m;
    depth = sdepth;
    while (b > a + 1) {
        int64_t pivot = (a + b) >> 1;
        model_probe(T, n, sa, P, m, pivot, la, lb, depth, d0, &c, &l, probes, chunks);
        depth++;
        if (c <= 0) {
            b = pivot;
            lb = l;
        } else {
            a = pivot;
            la = l;
        }
    }
    *lo = b;
    /* Upper bound in [split, R). */
    a = split;
    b = R;
    la = m;
    lb = lcpR;
    depth = sdepth;
    while (b > a + 1) {
        int64_t pivot = (a + b) >> 1;
        model_probe(T, n, sa, P, m, pivot, la, lb, depth, d0, &c, &l, probes, chunks);
        depth++;
        if (c < 0) {
            b = pivot;
            lb = l;
        } else {
            a = pivot;
            la = l;
        }
    }
    *hi = b;
}

/* ------------------------------------------------------------------ */
/* k-mer table (an exact shortcut for the top of the binary search)    */
/* ------------------------------------------------------------------ */

/* Compares suffix S_p with the k-base string X: -1 if S_p sorts before X
 * (including when S_p is a proper prefix of X), 0 if X is a prefix of S_p,
 * +1 otherwise. */
static int suffix_vs_string(const uint8_t *T, int64_t n, int64_t p, const uint8_t *X, int64_t k)
{
    for (int64_t t = 0; t < k; t++) {
        if (p + t >= n)
            return -1;
        if (T[p + t] != X[t])
            return T[p + t] < X[t] ? -1 : 1;
    }
    return 0;
}

/* The number of suffixes that sort before the k-base string whose bases are
 * the base-4 digits of x (A=0 C=1 G=2 T=3, most significant first), x in
 * [0, 4^k): the lower bound of that string in the sorted suffixes, by binary
 * search over sa. */
int64_t oracle_kmer_rank(const uint8_t *T, int64_t n, const int64_t *sa, int k, int64_t x)
{
    static const uint8_t letters[4] = {'A', 'C', 'G', 'T'};
    uint8_t X[32];
    for (int t = 0; t < k; t++)
        X[t] = letters[(x >> (2 * (k - 1 - t))) & 3];
    int64_t lo = 0, hi = n; /* first rank whose suffix is not before X */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (suffix_vs_string(T, n, sa[mid], X, k) < 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* table[x] = oracle_kmer_rank(x) for x in [0, 4^k); table[4^k] = n. */
void oracle_kmer_table(const uint8_t *T, int64_t n, const int64_t *sa, int k, int64_t *table)
{
    int64_t count = (int64_t)1 << (2 * k);
    for (int64_t x = 0; x < count; x++)
        table[x] = oracle_kmer_rank(T, n, sa, k, x);
    table[count] = n;
}

/* Byte model of the search as the CUDA path runs it on an index with a k-mer
 * table and 16-byte suffix records (measurement, not a parity output).
 * A query of m >= k bases starts between ranks table[x] - 1 and table[x + 1]
 * (x = its first k bases) and costs one table sector; shorter queries start
 * at [-1, n) and their first d0 probes are free (shared-memory key table).
 * Every other probe of the lockstep lower/upper-bound search reads one
 * 32-byte record sector holding the suffix's first 112 bases; a compare that
 * agrees on all 112 (m > 112, suffix >= 112 bases) also reads the 32-base
 * text windows from base 96 up to the one where it is decided.  *probes,
 * *windows count them; *table_reads is 1 or 0. */
/* The same model for one query given its k-mer bracket: has_bracket says
 * whether the query starts between ranks tlo - 1 and thi (tlo = table[x],
 * thi = table[x + 1] for its first k bases x), else it starts at [-1, n) with
 * its first d0 probes free. */
void oracle_probe_model_bracket(const uint8_t *T, int64_t n, const int64_t *sa, int has_bracket, int64_t tlo,
                                int64_t thi, int d0, const uint8_t *P, int64_t m, int64_t *probes,
                                int64_t *windows, int64_t *table_reads, int64_t *lo_out, int64_t *hi_out)
{
    *probes = 0;
    *windows = 0;
    *table_reads = 0;
    int64_t L = -1, R = n;
    int depth = 0, free_levels = 0;
    if (has_bracket) {
        L = tlo - 1;
        R = thi;
        *table_reads = 1;
    } else {
        free_levels = d0;
    }
    int phase = 0;
    int64_t HL = 0, HR = 0, lo = 0;
    for (;;) {
        if (R - L <= 1) {
            if (phase == 1) {
                lo = R;
                L = HL;
                R = HR;
                phase = 2;
                continue;
            }
            *lo_out = phase == 0 ? R : lo;
            *hi_out = R;
            return;
        }
        int64_t M = (L + R) >> 1;
        int64_t l;
        int c = query_cmp(T, n, sa[M], P, m, &l);
        if (depth >= free_levels) {
            (*probes)++;
            if (m > 112 && n - sa[M] >= 112 && l >= 112) {
                int64_t last = l < m - 1 ? l : m - 1;
                *windows += last / 32 - 3 + 1; /* windows from base 96 to the deciding one */
            }
        }
        depth++;
        if (c == 0 && phase == 0) {
            HL = M;
            HR = R;
            R = M;
            phase = 1;
        } else if (c < 0 || (c == 0 && phase == 1)) {
            R = M;
        } else {
            L = M;
        }
    }
}

void oracle_probe_model_kmer(const uint8_t *T, int64_t n, const int64_t *sa, const int64_t *table, int k,
                             int d0, const uint8_t *P, int64_t m, int64_t *probes, int64_t *windows,
                             int64_t *table_reads, int64_t *lo_out, int64_t *hi_out)
{
    int has = table && m >= k && k > 0;
    int64_t x = 0;
    if (has)
        for (int t = 0; t < k; t++)
            x = x * 4 + (P[t] == 'A' ? 0 : P[t] == 'C' ? 1 : P[t] == 'G' ? 2 : 3);
    oracle_probe_model_bracket(T, n, sa, has, has ? table[x] : 0, has ? table[x + 1] : 0, d0, P, m, probes,
                               windows, table_reads, lo_out, hi_out);
}
