// dc3_check.cpp -- runs the library's host DC3 construction (csrc/dc3_host.cpp)
// under AddressSanitizer and UndefinedBehaviorSanitizer.  The cases are every
// text over {A,C,G,T} of length <= 8, periodic and Fibonacci texts of lengths
// in each residue class mod 3, and seeded random texts.  Each is compared with
// std::sort of the suffixes under std::string order: A < C < G < T, and a
// proper prefix first.  The entry point's 64-bit output, its argument checks and
// its rejection of bytes outside the alphabet are also exercised.  Exit status
// 0 iff every check holds.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "dc3.h"
#include "sa.h"

static int failures = 0;

static void check(const std::string &t) {
    const size_t n = t.size();
    std::vector<uint32_t> got(n);
    const int st = sa::dc3_suffix_array(t.data(), n, got.data());
    std::vector<uint32_t> want(n);
    std::iota(want.begin(), want.end(), 0u);
    std::sort(want.begin(), want.end(),
              [&](uint32_t a, uint32_t b) { return t.compare(a, std::string::npos, t, b, std::string::npos) < 0; });
    if (st != SA_OK || got != want) {
        if (failures++ < 10) std::fprintf(stderr, "mismatch for a text of %zu bases: %.40s\n", n, t.c_str());
    }
}

int main() {
    const char acgt[] = "ACGT";
    for (int len = 1; len <= 8; len++)
        for (uint32_t c = 0; c < (1u << (2 * len)); c++) {
            std::string t(len, 'A');
            for (int i = 0; i < len; i++) t[i] = acgt[(c >> (2 * (len - 1 - i))) & 3];
            check(t);
        }
    const std::vector<std::string> units = {"A", "AC", "ACG", "AAC", "ACGT", "AACAG"};
    std::vector<size_t> lengths;
    for (size_t n = 9; n <= 60; n++) lengths.push_back(n);
    for (size_t n : {997, 998, 999, 3000, 3001, 3002}) lengths.push_back(n);
    for (const auto &u : units)
        for (size_t n : lengths) {
            std::string t;
            while (t.size() < n) t += u;
            t.resize(n);
            check(t);
        }
    std::string fa = "A", fb = "AC";
    while (fb.size() < 5000) {
        std::string next = fb + fa;
        fa = fb;
        fb = next;
    }
    for (size_t n : lengths) check(fb.substr(0, n));
    uint64_t s = 1303369200u;
    for (int rep = 0; rep < 6; rep++) {
        const size_t n = 20000 + rep;
        std::string t(n, 'A');
        for (size_t i = 0; i < n; i++) {
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            t[i] = acgt[s >> 62];
        }
        t.replace(n / 2, n / 5, t.substr(0, n / 5));  // a long exact repeat
        check(t);
    }

    // The C entry point: 64-bit output equals the 32-bit one; bad arguments and
    // bytes outside the alphabet are rejected.
    const std::string t = "acggtacgtac";
    std::vector<uint32_t> s32(t.size());
    std::vector<uint64_t> s64(t.size());
    bool ok = sa_suffix_array_host(t.data(), t.size(), 4, s32.data()) == SA_OK &&
              sa_suffix_array_host(t.data(), t.size(), 8, s64.data()) == SA_OK;
    for (size_t i = 0; ok && i < t.size(); i++) ok = s64[i] == s32[i];
    ok = ok && s32 == std::vector<uint32_t>({9, 0, 5, 10, 1, 6, 2, 7, 3, 8, 4});  // Table I
    ok = ok && sa_suffix_array_host(t.data(), 0, 4, s32.data()) == SA_ERR_ARG &&
         sa_suffix_array_host(t.data(), t.size(), 2, s32.data()) == SA_ERR_ARG &&
         sa_suffix_array_host(nullptr, t.size(), 4, s32.data()) == SA_ERR_ARG &&
         sa_suffix_array_host("ACNGT", 5, 4, s32.data()) == SA_ERR_BASE;
    if (!ok) failures++;
    if (failures)
        std::fprintf(stderr, "%d check(s) failed\n", failures);
    else
        std::printf("dc3 checks passed\n");
    return failures ? 1 : 0;
}
