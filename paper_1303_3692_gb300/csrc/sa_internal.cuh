// sa_internal.cuh -- layouts and device helpers shared by the libsa kernels.
//
// Packed text layout (Section III alphabet, order A < C < G < T):
//   base b of a sequence lives in 64-bit word b / 32 at bits
//   [63 - 2*(b % 32), 62 - 2*(b % 32)], codes A=0 C=1 G=2 T=3.  Big-endian
//   placement makes unsigned integer comparison of two aligned windows equal
//   to lexicographic comparison of their bases.  Bits past the end are zero
//   and every packed text carries SA_PAD_WORDS zero words after its last
//   word, so a 32-base window starting at any base < n reads in bounds.
//
// Packed queries: query q occupies 32-byte slots starting at slot
// ((q_offsets[q] - q_offsets[0]) >> 7) + q of the query word buffer (4 words
// per slot).  For consecutive queries the start grows by at least
// ceil(m_q / 128) slots, so no scan is needed to place them, and a query's
// first 128 bases sit in one aligned 32-byte sector.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sa.h"

#define SA_PAD_WORDS 2
#define SA_MAX_REFS 64
#define SA_MAX_KEY_DEPTH 14

namespace sa {

// Device view of one index, passed to the kernels.
struct RefDesc {
    const uint64_t *text;   // packed text, nwords + SA_PAD_WORDS words
    const void *sa;         // n entries of width 4 or 8
    const uint4 *keys;      // 2^depth key entries: 64 bases as two words (x,y = w0; z,w = w1)
    const uint8_t *keylen;  // 2^depth clamp lengths min(64, n - SA[rank])
    const uint4 *rec;       // 2n uint4: n 32-byte suffix records, see sa_index::rec
    const uint32_t *kmer;   // 4^kmer_k + 1 entries, see sa_index::kmer (null: none)
    uint64_t n;
    uint32_t depth;         // key-table depth d of this index; K = 2^d - 1 samples
    uint32_t smem_off;      // byte offset of this table in the search kernel's shared memory
    uint32_t use_depth;     // depth the search uses (<= depth); 0 = no table
    uint32_t kmer_k;        // k of the k-mer table (0: none)
};

// The compare outcome of the three cases of Section IV.
enum : int { CMP_LESS = -1, CMP_PREFIX = 0, CMP_GREATER = 1 };

__device__ __forceinline__ uint64_t ldg_u64(const uint64_t *p) { return __ldg(p); }

// 32 bases of the packed text starting at base position b (b < n + 32).
__device__ __forceinline__ uint64_t text_window(const uint64_t *__restrict__ T, uint64_t b) {
    const uint64_t w = b >> 5;
    const unsigned sh = (unsigned)(b & 31u) * 2u;
    const uint64_t a = ldg_u64(T + w);
    const uint64_t c = ldg_u64(T + w + 1);
    // (c >> 1) >> (63 - sh) is c >> (64 - sh) for sh > 0 and 0 for sh == 0.
    return (a << sh) | ((c >> 1) >> (63u - sh));
}

// Compares query P (packed words Q, length m >= 1) with the m-prefix of the
// suffix starting at text position p, beginning at base `start` (all bases
// before it are known equal; start < m).  Returns CMP_LESS if P sorts before
// the suffix, CMP_PREFIX if P is a prefix of it, CMP_GREATER if P sorts after
// it (a suffix that ends first sorts before P).  *lcp receives the common
// prefix length, capped at m.  Windows are 32 bases; the query side is read
// one aligned word at a time.
__device__ __forceinline__ int cmp_query_suffix(const uint64_t *__restrict__ T, uint64_t n, uint64_t p,
                                                const uint64_t *__restrict__ Q, uint32_t m,
                                                uint32_t start, uint32_t *lcp) {
    uint32_t off = start & ~31u;
    const int64_t avail0 = (int64_t)n - (int64_t)p;  // bases left in the suffix
    for (;;) {
        const int64_t avail = avail0 - (int64_t)off;
        const uint32_t qlen = min(32u, m - off);
        const uint32_t tlen = avail <= 0 ? 0u : (avail >= 32 ? 32u : (uint32_t)avail);
        const uint64_t q = __ldg(Q + (off >> 5));
        const uint64_t t = tlen ? text_window(T, p + off) : 0ull;
        const uint64_t x = q ^ t;
        const uint32_t d = x ? ((uint32_t)__clzll((long long)x) >> 1) : 32u;
        const uint32_t lim = min(qlen, tlen);
        if (d < lim) {
            *lcp = off + d;
            return q < t ? CMP_LESS : CMP_GREATER;
        }
        if (tlen < qlen) {
            *lcp = off + tlen;
            return CMP_GREATER;
        }
        if (off + 32u >= m) {
            *lcp = m;
            return CMP_PREFIX;
        }
        off += 32u;
    }
}

// Base code of an ASCII byte; returns 4 for a byte outside {ACGTacgt}.
__device__ __forceinline__ uint32_t base_code(uint32_t c) {
    const uint32_t u = c & 0xDFu;  // fold lower case
    const uint32_t x = (u >> 1) & 3u;  // A:0 C:1 G:3 T:2
    const uint32_t code = x ^ (x >> 1);  // A:0 C:1 G:2 T:3
    const bool ok = (u == 'A') | (u == 'C') | (u == 'G') | (u == 'T');
    return ok ? code : 4u;
}

// First 32-byte slot of a query whose bases start at byte a_rel of the batch.
__host__ __device__ __forceinline__ uint64_t query_slot(uint64_t a_rel, uint64_t q) { return (a_rel >> 7) + q; }

// Per-query record written by the pack kernel for the search, 32 bytes (two
// uint4): x, y = the starting bracket (L, R) of the binary search
// (L = 0xFFFFFFFF for -1), z = m (kQueryInvalid for a query that cannot be
// searched), w = its first slot; then the query's first two packed words
// (bases 0-63), so that the search starts from one sector.
constexpr uint32_t kQueryInvalid = 0xFFFFFFFFu;

// Four ASCII bytes (little-endian in v) to four 2-bit codes in the low byte,
// first base in the top two bits.  Per byte, with u the case-folded byte:
// x = (u >> 1) & 3 is A0 C1 G3 T2 and c = x ^ (x >> 1) is A0 C1 G2 T3.  The
// codes sit at bits 0, 8, 16, 24; one multiply by 2^30 + 2^20 + 2^10 + 1
// moves them to bits 30, 28, 26, 24 without carries between the partial
// products.  The check rebuilds each letter from its code, 'A' + 2c + 2h +
// 11 (c & h) with h = c >> 1 (giving A, C, G, T for c = 0..3), and ORs any
// difference from u into *bad.
__device__ __forceinline__ uint32_t pack4_fast(uint32_t v, uint32_t *bad) {
    const uint32_t u = v & 0xDFDFDFDFu;
    const uint32_t x = (u >> 1) & 0x03030303u;
    const uint32_t h0 = (x >> 1) & 0x01010101u;
    const uint32_t c = x ^ h0;                     // per byte: A0 C1 G2 T3
    const uint32_t h = (c >> 1) & 0x01010101u;
    const uint32_t expect = 0x41414141u + 2u * c + 2u * h + 11u * (c & h);
    *bad |= u ^ expect;
    return (c * 0x40100401u) >> 24;
}

// Packs the 32 ASCII bases starting at byte s of a (the first nb <= 32 belong
// to the query; the rest pack as A).  When nine aligned 32-bit words around
// them lie inside [a, a + total) they are read and aligned with funnel
// shifts; the check covers only the query's own nb bytes.  Otherwise (the
// batch's last bytes) the bytes are read one at a time.  Returns the word;
// *bad becomes non-zero if one of the nb bytes is not a base.
__device__ __forceinline__ uint64_t pack_word(const uint8_t *__restrict__ a, uint64_t total, uint64_t s,
                                              uint32_t nb, uint32_t *bad) {
    const uintptr_t lo_addr = ((uintptr_t)(a + s)) & ~(uintptr_t)3;
    uint64_t word = 0;
    if (lo_addr >= (uintptr_t)a && lo_addr + 36 <= (uintptr_t)(a + total)) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(lo_addr);
        const uint32_t sh = (uint32_t)(((uintptr_t)(a + s)) & 3u) * 8u;
        uint32_t v[9];
#pragma unroll
        for (int i = 0; i < 9; i++) v[i] = __ldg(p + i);
        uint32_t hi = 0, lo = 0, b = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint32_t gb = 0;
            const uint32_t g = pack4_fast(__funnelshift_r(v[i], v[i + 1], sh), &gb);
            const int own = (int)nb - 4 * i;  // bytes of this group that belong to the query
            b |= own >= 4 ? gb : (own > 0 ? gb & ((1u << (8 * own)) - 1u) : 0u);
            if (i < 4)
                hi = (hi << 8) | g;
            else
                lo = (lo << 8) | g;
        }
        *bad |= b;
        word = ((uint64_t)hi << 32) | lo;
        if (nb < 32) word &= ~0ull << (64u - 2u * nb);
    } else {
        for (uint32_t j = 0; j < 32; j++) {
            uint32_t code = 0;
            if (j < nb) {
                code = base_code(a[s + j]);
                if (code > 3) {
                    *bad |= 1u;
                    code = 0;
                }
            }
            word = (word << 2) | code;
        }
    }
    return word;
}

// One 32-byte (one DRAM sector) read-only load; p must be 32-byte aligned.
// A single request per sector instead of two 16-byte ones, which the memory
// system would otherwise serve as two misses.
__device__ __forceinline__ void ldg32(const void *p, uint4 *lo, uint4 *hi) {
    unsigned long long a, b, c, d;
    asm volatile("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
    *lo = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    *hi = make_uint4((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)d, (uint32_t)(d >> 32));
}

template <typename IdxT>
__device__ __forceinline__ uint64_t sa_at(const void *sa, uint64_t i) {
    return (uint64_t)__ldg(reinterpret_cast<const IdxT *>(sa) + i);
}

}  // namespace sa

// ---------------------------------------------------------------------------
// Host-side internals shared by the translation units.
// ---------------------------------------------------------------------------
struct sa_index {
    uint64_t n;
    uint32_t width;      // 4 or 8
    uint32_t depth;      // key-table depth
    int device;
    uint64_t nwords;     // packed words without padding
    uint64_t *text;      // device
    void *sa;            // device
    uint4 *keys;         // device, 2^depth entries
    uint8_t *keylen;     // device, 2^depth entries
    uint4 *rec;          // device, n 32-byte records in suffix-array order (2 uint4 each):
                         // the first 112 bases of suffix SA[i] as packed words w0, w1, w2
                         // (bases 0-95) and the 16 bases 96-111 in the high-to-low bits of a
                         // 32-bit word, then SA[i]: {w0.lo, w0.hi, w1.lo, w1.hi}, {w2.lo,
                         // w2.hi, w3, SA[i]}
    uint32_t *kmer;      // device, 4^kmer_k + 1 entries: kmer[x] = number of suffixes that
                         // sort before the k-base string x (x as a 2k-bit number); null if none
    uint32_t kmer_k;
    uint64_t device_bytes;
};

namespace sa {

int status_from_cuda(cudaError_t e);
cudaMemPool_t scratch_pool(int device);
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s);
void scratch_free(void *p, cudaStream_t s);
int device_sm_count();

// Kernels launched from the API translation unit.
cudaError_t launch_pack_text(const char *ascii, uint64_t n, uint64_t *words, uint64_t nwords_padded,
                             int *err_flag, cudaStream_t s);
struct SearchLaunch;
cudaError_t launch_pack_queries(const SearchLaunch &L, int *err_flag, cudaStream_t s);
int build_suffix_array(sa_index *idx, cudaStream_t s);
cudaError_t launch_build_keys(sa_index *idx, cudaStream_t s);
cudaError_t launch_build_records(sa_index *idx, cudaStream_t s);
cudaError_t launch_build_kmer(sa_index *idx, cudaStream_t s);

// Descriptors of every index a call uses, passed by value as a kernel
// parameter (64 x 72 bytes; kernel parameters may take up to 32 KB).
struct RefTable {
    RefDesc r[SA_MAX_REFS];
};

struct SearchLaunch {
    RefTable refs;
    uint32_t n_refs;
    uint32_t width;
    const char *ascii;        // query bases, indexed by q_off[q] - first
    uint64_t *qwords;         // packed queries (written by the pack kernel)
    const uint64_t *q_off;    // n_q + 1 offsets
    uint64_t first;           // q_off[0]
    uint64_t total;           // q_off[n_q] - q_off[0]: query ranges past it are invalid
    const uint32_t *q_ref;    // null when n_refs == 1
    uint64_t n_q;
    uint4 *meta;              // 2 n_q uint4: per-query records written by the pack kernel
    sa_result *out;
    int *pack_err;            // device flag: some query had a non-ACGT byte or bad offsets
    unsigned long long *counter;
    int *status;
    uint32_t smem_bytes;      // shared-memory key tables
    uint32_t threads, blocks, chunk;
};
cudaError_t launch_search(const SearchLaunch &L, cudaStream_t s);
cudaError_t launch_search_plain(const SearchLaunch &L, cudaStream_t s);
uint32_t search_table_bytes(uint32_t depth);  // shared-memory bytes of a depth-d key table

struct LocateLaunch {
    RefTable refs;
    uint32_t n_refs, width;
    const uint32_t *q_ref;
    const sa_result *res;
    uint64_t n_q;
    uint32_t cap;
    uint64_t *out_offsets;
    void *out_pos;
    uint64_t capacity;
    uint64_t *partials;       // scratch: one entry per scan tile + 1
};
uint64_t locate_tiles(uint64_t n_q);
// Device address of the static scratch of sa_locate_noalloc on the current
// device (looked up once per device) and the number of partial sums it holds.
cudaError_t locate_static_partials(uint64_t **ptr, uint64_t *entries);
cudaError_t launch_locate(const LocateLaunch &L, cudaStream_t s);

}  // namespace sa
