// dc3_host.cpp -- the suffix array by the construction Section III describes:
// the difference cover modulo 3 (DC3, the skew algorithm of Kärkkäinen and
// Sanders, 2003), run on the host CPU as the paper runs it.
//
// One level of the recursion, for a string s[0..n) over [1, K] followed by
// three zeros (a zero sorts before every letter, so a suffix that is a proper
// prefix of another sorts first, as in Table I):
//   1. The sample suffixes start at i mod 3 != 0 (Table II ranks them).  When
//      n mod 3 == 1 the empty suffix at i = n joins the sample, so that the
//      mod-1 part of the reduced string ends in a unique letter.
//   2. Radix-sort the samples by their first three letters and name each
//      distinct triple by its rank.  The reduced string lists the names of the
//      mod-1 samples in text order, then those of the mod-2 samples.  If two
//      samples share a name, its suffix array (recursively) orders them.
//   3. Sort the suffixes at i mod 3 == 0 by (s[i], rank of the sample at i+1);
//      Section III's example orders B0 = {0, 3, 6, 9} this way, S9 <= S0 <=
//      S6 <= S3.
//   4. Merge the two sorted lists.  A mod-0 suffix and a sample compare by at
//      most two letters and one sample rank.
// Every step is linear, so one level costs O(n) and the whole recursion O(n).
#include "dc3.h"

#include <new>
#include <vector>

#include "sa.h"

namespace sa {
namespace {

// Stable counting sort of in[0..m) into out[0..m) by key(p) in [0, K].
template <typename KeyFn>
void counting_sort(const uint32_t *in, uint32_t *out, size_t m, uint32_t K, KeyFn key, std::vector<uint32_t> &cnt) {
    cnt.assign((size_t)K + 1, 0);
    for (size_t t = 0; t < m; t++) cnt[key(in[t])]++;
    uint32_t sum = 0;
    for (size_t c = 0; c <= K; c++) {
        const uint32_t here = cnt[c];
        cnt[c] = sum;
        sum += here;
    }
    for (size_t t = 0; t < m; t++) out[cnt[key(in[t])]++] = in[t];
}

// Suffix array of s[0..n) (letters in [1, K], s[n] = s[n+1] = s[n+2] = 0)
// into sa[0..n).  Throws std::bad_alloc.
template <typename C>
void skew(const C *s, size_t n, uint32_t K, uint32_t *sa) {
    const size_t n0 = (n + 2) / 3;  // positions 0 mod 3; also the mod-1 samples, with the empty one
    const size_t n2 = n / 3;        // mod-2 samples
    const size_t n02 = n0 + n2;
    // Index of sample position p in the reduced string.
    auto ridx = [n0](size_t p) { return p % 3 == 1 ? (p - 1) / 3 : n0 + (p - 2) / 3; };

    // Step 2: sort the samples by their leading triple.
    std::vector<uint32_t> cnt;
    std::vector<uint32_t> red(n02 + 3, 0);  // the reduced string, then the sample ranks
    {
        std::vector<uint32_t> a(n02), b(n02);
        for (size_t j = 0; j < n0; j++) a[j] = (uint32_t)(3 * j + 1);
        for (size_t j = 0; j < n2; j++) a[n0 + j] = (uint32_t)(3 * j + 2);
        counting_sort(a.data(), b.data(), n02, K, [s](uint32_t p) { return (uint32_t)s[(size_t)p + 2]; }, cnt);
        counting_sort(b.data(), a.data(), n02, K, [s](uint32_t p) { return (uint32_t)s[(size_t)p + 1]; }, cnt);
        counting_sort(a.data(), b.data(), n02, K, [s](uint32_t p) { return (uint32_t)s[p]; }, cnt);
        uint32_t names = 0;
        size_t prev = SIZE_MAX;
        for (size_t t = 0; t < n02; t++) {
            const size_t p = b[t];
            if (prev == SIZE_MAX || s[p] != s[prev] || s[p + 1] != s[prev + 1] || s[p + 2] != s[prev + 2]) names++;
            red[ridx(p)] = names;
            prev = p;
        }
        if (names < n02) {
            // Equal triples: order the samples by the suffixes of the reduced string.
            std::vector<uint32_t>().swap(a);
            std::vector<uint32_t>().swap(b);
            std::vector<uint32_t> sar(n02);
            skew(red.data(), n02, names, sar.data());
            for (size_t r = 0; r < n02; r++) red[sar[r]] = (uint32_t)(r + 1);
        }
        // Otherwise each name already is its sample's rank.
    }
    // Rank (1-based) of the sample suffix at position p; 0 for the empty
    // suffix and beyond, which sort before every nonempty one.
    auto rank = [&](size_t p) -> uint32_t { return p >= n ? 0u : red[ridx(p)]; };

    // The samples in sorted order (the empty one included, at the front).
    std::vector<uint32_t> s12(n02);
    for (size_t j = 0; j < n02; j++) {
        const uint32_t r = red[j];
        s12[r - 1] = (uint32_t)(j < n0 ? 3 * j + 1 : 3 * (j - n0) + 2);
    }

    // Step 3: the mod-1 samples in rank order give their predecessors sorted by
    // the rank of i+1; a stable sort by s[i] finishes the order.
    std::vector<uint32_t> s0(n0), t0(n0);
    {
        size_t k = 0;
        for (size_t r = 0; r < n02; r++)
            if (s12[r] % 3 == 1) t0[k++] = s12[r] - 1;
        counting_sort(t0.data(), s0.data(), n0, K, [s](uint32_t p) { return (uint32_t)s[p]; }, cnt);
    }
    std::vector<uint32_t>().swap(t0);

    // Step 4: merge.  Is the mod-0 suffix i before the sample suffix j?
    auto before = [&](size_t i, size_t j) -> bool {
        if (s[i] != s[j]) return s[i] < s[j];
        if (j % 3 == 1) return rank(i + 1) < rank(j + 1);
        if (s[i + 1] != s[j + 1]) return s[i + 1] < s[j + 1];
        return rank(i + 2) < rank(j + 2);
    };
    size_t a = 0, b = (n02 > 0 && s12[0] >= n) ? 1 : 0, out = 0;  // b skips the empty sample
    while (a < n0 && b < n02) {
        if (before(s0[a], s12[b]))
            sa[out++] = s0[a++];
        else
            sa[out++] = s12[b++];
    }
    while (a < n0) sa[out++] = s0[a++];
    while (b < n02) sa[out++] = s12[b++];
}

}  // namespace

int dc3_suffix_array(const char *text, uint64_t n, uint32_t *sa) {
    try {
        std::vector<uint8_t> s((size_t)n + 3, 0);
        for (uint64_t i = 0; i < n; i++) {
            switch (text[i]) {
                case 'A': case 'a': s[i] = 1; break;
                case 'C': case 'c': s[i] = 2; break;
                case 'G': case 'g': s[i] = 3; break;
                case 'T': case 't': s[i] = 4; break;
                default: return SA_ERR_BASE;
            }
        }
        skew(s.data(), (size_t)n, 4u, sa);
    } catch (const std::bad_alloc &) {
        return SA_ERR_NOMEM;
    }
    return SA_OK;
}

}  // namespace sa

extern "C" int sa_suffix_array_host(const char *text, uint64_t n, uint32_t width, void *sa_out) {
    if (!text || !sa_out || n == 0 || n >= 0xFFFFFFFFull || (width != 4 && width != 8)) return SA_ERR_ARG;
    if (width == 4) return sa::dc3_suffix_array(text, n, static_cast<uint32_t *>(sa_out));
    uint32_t *tmp = new (std::nothrow) uint32_t[n];
    if (!tmp) return SA_ERR_NOMEM;
    const int st = sa::dc3_suffix_array(text, n, tmp);
    if (st == SA_OK) {
        uint64_t *dst = static_cast<uint64_t *>(sa_out);
        for (uint64_t i = 0; i < n; i++) dst[i] = tmp[i];
    }
    delete[] tmp;
    return st;
}
