/*
 * oracle_check.c -- drives every routine of oracle/oracle.c on small cases so
 * that AddressSanitizer and UndefinedBehaviorSanitizer see each code path.
 * The cases are every text over {A,C,G,T} of length <= 6 with every query of
 * length <= 3 plus longer ones, and seeded repetitive texts searched in
 * threaded batches.  It cross-checks the routines against one another: Alg. 1
 * against the definition count, counts against brute force, the located
 * positions, the k-mer table's brackets and the byte models' intervals.
 * Exit status 0 iff every check holds.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_normalize(const uint8_t *in, int64_t n, uint8_t *out, int64_t *bad);
void oracle_sa_naive(const uint8_t *T, int64_t n, int64_t *sa);
void oracle_ranks(const int64_t *sa, int64_t n, int64_t *rank1);
int oracle_verify_sa(const uint8_t *T, int64_t n, const int64_t *sa, int nthreads, int64_t *where);
void oracle_search(const uint8_t *T, int64_t n, const int64_t *sa, const uint8_t *P, int64_t m, int64_t *lo,
                   int64_t *hi);
void oracle_rank_count(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m, int64_t *lo, int64_t *hi);
int64_t oracle_bruteforce(const uint8_t *T, int64_t n, const uint8_t *P, int64_t m, int64_t *pos, int64_t cap);
void oracle_sort_positions(const uint8_t *T, int64_t n, int64_t *pos, int64_t k);
void oracle_search_batch(const uint8_t *T, int64_t n, const int64_t *sa, const uint8_t *Q, const int64_t *qoff,
                         int64_t nq, int64_t *lo, int64_t *hi, int nthreads);
void oracle_rank_count_batch(const uint8_t *T, int64_t n, const uint8_t *Q, const int64_t *qoff, int64_t nq,
                             int64_t *lo, int64_t *hi, int nthreads);
void oracle_locate(const int64_t *sa, int64_t lo, int64_t hi, int64_t cap, int64_t *out);
void oracle_probe_model(const uint8_t *T, int64_t n, const int64_t *sa, const uint8_t *P, int64_t m, int d0,
                        int64_t *probes, int64_t *chunks, int64_t *lo, int64_t *hi);
void oracle_kmer_table(const uint8_t *T, int64_t n, const int64_t *sa, int k, int64_t *table);
void oracle_probe_model_kmer(const uint8_t *T, int64_t n, const int64_t *sa, const int64_t *table, int k, int d0,
                             const uint8_t *P, int64_t m, int64_t *probes, int64_t *windows, int64_t *table_reads,
                             int64_t *lo_out, int64_t *hi_out);

static int failures = 0;

#define CHECK(cond, ...)                         \
    do {                                         \
        if (!(cond)) {                           \
            if (failures++ < 10) {               \
                fprintf(stderr, __VA_ARGS__);    \
                fputc('\n', stderr);             \
            }                                    \
        }                                        \
    } while (0)

static const uint8_t ACGT[4] = {'A', 'C', 'G', 'T'};

static void fill_word(uint8_t *dst, int64_t len, int64_t code)
{
    for (int64_t t = len - 1; t >= 0; t--) {
        dst[t] = ACGT[code & 3];
        code >>= 2;
    }
}

/* One text against one query: every routine that takes a single query. */
static void check_query(const uint8_t *T, int64_t n, const int64_t *sa, const int64_t *table, int k,
                        const uint8_t *P, int64_t m)
{
    int64_t lo, hi, lo2, hi2;
    oracle_search(T, n, sa, P, m, &lo, &hi);
    oracle_rank_count(T, n, P, m, &lo2, &hi2);
    CHECK(lo == lo2 && hi == hi2, "search [%lld,%lld) vs definition [%lld,%lld) n=%lld m=%lld", (long long)lo,
          (long long)hi, (long long)lo2, (long long)hi2, (long long)n, (long long)m);
    int64_t pos[64];
    int64_t cnt = m ? oracle_bruteforce(T, n, P, m, pos, 64) : n;
    CHECK(cnt == hi - lo, "brute force %lld vs %lld", (long long)cnt, (long long)(hi - lo));
    if (m && cnt <= 64) {
        int64_t loc[64];
        oracle_locate(sa, lo, hi, 64, loc);
        oracle_sort_positions(T, n, pos, cnt);
        CHECK(memcmp(loc, pos, (size_t)cnt * sizeof(int64_t)) == 0, "located positions differ");
    }
    int64_t probes = 0, chunks = 0, plo, phi;
    oracle_probe_model(T, n, sa, P, m, 0, &probes, &chunks, &plo, &phi);
    CHECK(plo == lo && phi == hi, "probe model interval differs");
    int64_t windows = 0, reads = 0;
    probes = 0;
    oracle_probe_model_kmer(T, n, sa, table, k, 0, P, m, &probes, &windows, &reads, &plo, &phi);
    CHECK(plo == lo && phi == hi, "k-mer probe model interval differs (k=%d m=%lld)", k, (long long)m);
}

static void check_text(const uint8_t *T, int64_t n, const uint8_t *Q, const int64_t *qoff, int64_t nq)
{
    int64_t *sa = malloc((size_t)n * sizeof(int64_t));
    int64_t *rank1 = malloc((size_t)n * sizeof(int64_t));
    oracle_sa_naive(T, n, sa);
    int64_t where = 0;
    CHECK(oracle_verify_sa(T, n, sa, 1, &where) == 0, "verify failed at %lld", (long long)where);
    CHECK(oracle_verify_sa(T, n, sa, 3, &where) == 0, "threaded verify failed at %lld", (long long)where);
    oracle_ranks(sa, n, rank1);
    for (int64_t k = 0; k < n; k++)
        CHECK(rank1[sa[k]] == k + 1, "rank does not invert the suffix array");
    int k = n < 16 ? 1 : n < 256 ? 2 : 3;
    int64_t *table = malloc((((size_t)1 << (2 * k)) + 1) * sizeof(int64_t));
    oracle_kmer_table(T, n, sa, k, table);
    for (int64_t x = 0; x < ((int64_t)1 << (2 * k)); x++)
        CHECK(table[x] <= table[x + 1], "k-mer table not monotone");
    for (int64_t q = 0; q < nq; q++)
        check_query(T, n, sa, table, k, Q + qoff[q], qoff[q + 1] - qoff[q]);
    free(table);
    free(rank1);
    free(sa);
}

int main(void)
{
    /* Queries: every string of length <= 3 (with the empty one) and a few longer. */
    enum { MAXQ = 128 };
    uint8_t Q[MAXQ * 12];
    int64_t qoff[MAXQ + 1];
    int64_t nq = 0, used = 0;
    qoff[0] = 0;
    for (int64_t len = 0; len <= 3; len++)
        for (int64_t c = 0; c < ((int64_t)1 << (2 * len)); c++) {
            fill_word(Q + used, len, c);
            used += len;
            qoff[++nq] = used;
        }
    const char *longer[] = {"ACGTACG", "AAAAAAAA", "CGTACGTA", "TTTTTTTTTTT"};
    for (int i = 0; i < 4; i++) {
        size_t L = strlen(longer[i]);
        memcpy(Q + used, longer[i], L);
        used += (int64_t)L;
        qoff[++nq] = used;
    }

    /* Every text of length 1..6. */
    uint8_t T[8];
    for (int64_t n = 1; n <= 6; n++)
        for (int64_t c = 0; c < ((int64_t)1 << (2 * n)); c++) {
            fill_word(T, n, c);
            check_text(T, n, Q, qoff, nq);
        }

    /* Case folding and a rejected byte. */
    uint8_t in[6] = {'a', 'c', 'G', 't', 'N', 'A'}, out[6];
    int64_t bad = -1;
    CHECK(oracle_normalize(in, 4, out, &bad) == 0 && memcmp(out, "ACGT", 4) == 0, "normalize failed");
    CHECK(oracle_normalize(in, 6, out, &bad) == -1 && bad == 4, "normalize missed the N");

    /* Seeded repetitive texts, batches searched on several threads. */
    uint64_t s = 1303369200u;
    for (int rep = 0; rep < 4; rep++) {
        int64_t n = 3000 + rep;
        uint8_t *R = malloc((size_t)n);
        for (int64_t i = 0; i < n; i++) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            R[i] = ACGT[s >> 62];
        }
        memcpy(R + n / 2, R, (size_t)(n / 4)); /* a long exact repeat */
        for (int64_t i = 100; i < 400; i++)    /* a tandem run */
            R[i] = ACGT[(i % 3) & 3];
        int64_t bq = 400, *boff = malloc((size_t)(bq + 1) * sizeof(int64_t));
        uint8_t *B = malloc((size_t)bq * 40);
        boff[0] = 0;
        for (int64_t q = 0; q < bq; q++) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            int64_t len = (int64_t)(s >> 59) + 1; /* 1..32 */
            int64_t at = (int64_t)((s >> 20) % (uint64_t)(n - len));
            memcpy(B + boff[q], R + at, (size_t)len);
            if (q % 3 == 0)
                B[boff[q] + len / 2] = ACGT[(s >> 8) & 3];
            boff[q + 1] = boff[q] + len;
        }
        int64_t *sa = malloc((size_t)n * sizeof(int64_t));
        int64_t *lo = malloc((size_t)bq * sizeof(int64_t)), *hi = malloc((size_t)bq * sizeof(int64_t));
        int64_t *lo2 = malloc((size_t)bq * sizeof(int64_t)), *hi2 = malloc((size_t)bq * sizeof(int64_t));
        oracle_sa_naive(R, n, sa);
        int64_t where = 0;
        CHECK(oracle_verify_sa(R, n, sa, 4, &where) == 0, "repetitive text: verify failed");
        oracle_search_batch(R, n, sa, B, boff, bq, lo, hi, 4);
        oracle_rank_count_batch(R, n, B, boff, bq, lo2, hi2, 3);
        for (int64_t q = 0; q < bq; q++)
            CHECK(lo[q] == lo2[q] && hi[q] == hi2[q], "batch search differs from definition at %lld",
                  (long long)q);
        free(hi2);
        free(lo2);
        free(hi);
        free(lo);
        free(sa);
        free(B);
        free(boff);
        free(R);
    }
    if (failures)
        fprintf(stderr, "%d check(s) failed\n", failures);
    else
        printf("oracle checks passed\n");
    return failures ? 1 : 0;
}
