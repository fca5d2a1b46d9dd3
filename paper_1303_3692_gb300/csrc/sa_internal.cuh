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
// Packed query batch: the bases of a whole batch (q_offsets[0] ..
// q_offsets[n_q]) packed like a text, 32 per word, with SA_TQ_PAD_WORDS zero
// words after the last, and one 32-bit mask per word whose bit i marks base
// 32 w + i as not in {A,C,G,T,a,c,g,t}.  Query q's bases start at base
// q_offsets[q] - q_offsets[0], so any of its 32-base windows is one
// text_window read.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sa.h"

#define SA_PAD_WORDS 2
#define SA_TQ_PAD_WORDS 6
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
    const uint4 *krt;       // 4^kmer_k 64-byte k-mer entries, see sa_index::krt (null: none)
    uint64_t n;
    uint32_t depth;         // key-table depth d of this index; K = 2^d - 1 samples
    uint32_t smem_off;      // byte offset of this table in the search kernel's shared memory
    uint32_t use_depth;     // depth the search uses (<= depth); 0 = no table
    uint32_t kmer_k;        // k of the k-mer table (0: none)
    uint64_t kbase;         // k-mer entries of the earlier indexes of the call (k-mer order buckets)
};

// k-mer order of a batch (bucket.cu): the slices of the k-mer entries of a
// call's indexes, plus one bucket for queries without a k-mer bracket.
constexpr uint32_t kNumBuckets = 256;
// The k-mer-ordered list's 64-byte records (bucket.cu writes, front.cu reads):
//   {m, q, qa.lo, qa.hi | ref << 16 | kListNeedsEntry}  length, index, first
//       base in the packed batch (qa < 2^48), reference id (< 2^15), and
//       whether the query has a k-mer bracket to read
//   {w0, w1}, {w2, w3}, {w4, w5}  its first 192 bases as packed words (the
//       words past the query's end are not its bases)
constexpr uint32_t kListNeedsEntry = 0x80000000u;
constexpr uint64_t kListMaxBase = 1ull << 48;
// The list's plan (bucket.cu), 32-bit words: every kListSampleStride-th
// query's bucket counted; from those counts each bucket's region of the list
// (start, capacity) and a cursor; after the scatter, the exclusive prefix
// sums of the regions' fills (kNumBuckets + 2 words, the last the sum); and
// the overflow region that takes what does not fit a bucket's region.
constexpr uint32_t kListSampleStride = 32;
constexpr uint32_t kPlanSample = 0;
constexpr uint32_t kPlanStart = kPlanSample + kNumBuckets + 1;
constexpr uint32_t kPlanCap = kPlanStart + kNumBuckets + 1;
constexpr uint32_t kPlanCursor = kPlanCap + kNumBuckets + 1;
constexpr uint32_t kPlanPrefix = kPlanCursor + kNumBuckets + 1;
constexpr uint32_t kPlanOvStart = kPlanPrefix + kNumBuckets + 2;
constexpr uint32_t kPlanOvCursor = kPlanOvStart + 1;
constexpr uint32_t kPlanWords = kPlanOvCursor + 1;
// Records the list needs room for, at most: every bucket's region (the sample
// counts scaled up by 9/8, plus 256) and an overflow region for every query.
__host__ __device__ constexpr uint64_t list_capacity(uint64_t n_q) {
    return (n_q + kListSampleStride) * 9 / 8 + 256ull * (kNumBuckets + 1) + n_q;
}

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

// Base code of an ASCII byte; returns 4 for a byte outside {ACGTacgt}.
__device__ __forceinline__ uint32_t base_code(uint32_t c) {
    const uint32_t u = c & 0xDFu;  // fold lower case
    const uint32_t x = (u >> 1) & 3u;  // A:0 C:1 G:3 T:2
    const uint32_t code = x ^ (x >> 1);  // A:0 C:1 G:2 T:3
    const bool ok = (u == 'A') | (u == 'C') | (u == 'G') | (u == 'T');
    return ok ? code : 4u;
}

// Marks a query that cannot be searched (a byte that is not a base,
// inconsistent offsets or an out-of-range reference id).
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

// q_ref bit 31 under SA_PARAM_STRAND_PER_QUERY: search the query's reverse complement.
constexpr uint32_t kStrandBit = 0x80000000u;

// A query's first base in the packed batch tq: its own range [qa, qe), or
// for the other strand the mirrored range of the reverse-complement packing,
// which starts at base rc_base of tq (base i of that packing is the
// complement of batch base total - 1 - i).
__device__ __forceinline__ uint64_t strand_start(uint64_t qa, uint64_t qe, uint64_t total, bool rc,
                                                 uint64_t rc_base) {
    return rc ? rc_base + (total - qe) : qa;
}

// Bits [lo, hi) of a 32-bit mask (0 <= lo <= hi <= 32).
__device__ __forceinline__ uint32_t bit_range(uint32_t lo, uint32_t hi) {
    const uint32_t upto = hi >= 32u ? 0xFFFFFFFFu : ((1u << hi) - 1u);
    return upto & ~((1u << lo) - 1u);
}

// The head of a query of the packed batch: its first 128 bases as four
// packed words w[0..3] (base 0 in the top bits of w[0]; bits past the query
// hold the batch's next bases), read as five words from word w_lo = qa / 32
// of tq with the shift of qa % 32.  With check set, returns whether all m
// bases (from bit qa % 32 of word w_lo on) are marked valid in the per-word
// masks tv; else returns true without reading the masks.
__device__ __forceinline__ bool load_query_head(const uint64_t *__restrict__ tq, const uint32_t *__restrict__ tv,
                                                uint64_t w_lo, uint32_t b0, uint32_t m, bool check,
                                                uint64_t w[4]) {
    const uint32_t sh = b0 * 2u;
    uint64_t t[5];
#pragma unroll
    for (int i = 0; i < 5; i++) t[i] = __ldg(tq + w_lo + i);
#pragma unroll
    for (int j = 0; j < 4; j++) w[j] = (t[j] << sh) | ((t[j + 1] >> 1) >> (63u - sh));
    if (!check) return true;
    uint32_t v[5];
#pragma unroll
    for (int i = 0; i < 5; i++) v[i] = __ldg(tv + w_lo + i);
    uint32_t badbits = 0;
    const uint64_t end = (uint64_t)b0 + m;  // one past the query's last bit, from word w_lo
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const uint32_t lo = i == 0 ? b0 : 0u;
        const uint64_t wend = 32ull * (i + 1);
        const uint32_t hi = end >= wend ? 32u : (end > 32ull * i ? (uint32_t)(end - 32ull * i) : 0u);
        if (hi > lo) badbits |= v[i] & bit_range(lo, hi);
    }
    for (uint64_t i = 5; 32ull * i < end; i++) {  // queries longer than 128 bases
        const uint32_t hi = end >= 32ull * (i + 1) ? 32u : (uint32_t)(end - 32ull * i);
        badbits |= __ldg(tv + w_lo + i) & bit_range(0, hi);
    }
    return badbits == 0;
}

// One query's result, written as one 32-byte store (a whole DRAM sector, so a
// result at a random slot needs no read-modify-write): [lo, hi), count and
// flags; lo = ~0 marks an invalid query (all-ones result).  trunc_cap: the
// call's locate cap (a count above it sets SA_RESULT_TRUNCATED), or ~0u.
__device__ __forceinline__ void store_result(sa_result *out, uint64_t q, uint64_t lo, uint64_t hi,
                                             uint32_t trunc_cap) {
    const bool bad = lo == ~0ull;
    const uint64_t count = bad ? ~0ull : hi - lo;
    const uint64_t flags = bad ? (uint64_t)SA_RESULT_INVALID
                               : (count > (uint64_t)trunc_cap ? (uint64_t)SA_RESULT_TRUNCATED : 0ull);
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(out + q), "l"(lo), "l"(hi), "l"(count),
                 "l"(flags)
                 : "memory");
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

// Predicated read-only loads: when pred is false nothing is read and the
// outputs keep their values.  p must be 32-byte (ldg32_if) or 16-byte
// (ldg16_if) aligned when pred is true.
__device__ __forceinline__ void ldg32_if(bool pred, const void *p, uint4 *lo, uint4 *hi) {
    unsigned long long a = 0, b = 0, c = 0, d = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t"
        "@p ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];\n\t}"
        : "+l"(a), "+l"(b), "+l"(c), "+l"(d)
        : "l"(p), "r"((uint32_t)pred));
    *lo = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    *hi = make_uint4((uint32_t)c, (uint32_t)(c >> 32), (uint32_t)d, (uint32_t)(d >> 32));
}

__device__ __forceinline__ void ldg16_if(bool pred, const void *p, uint64_t *x, uint64_t *y) {
    unsigned long long a = 0, b = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %3, 0;\n\t"
        "@p ld.global.nc.v2.u64 {%0, %1}, [%2];\n\t}"
        : "+l"(a), "+l"(b)
        : "l"(p), "r"((uint32_t)pred));
    *x = a;
    *y = b;
}

// One window of a compare: q and t hold qlen and tlen bases (tlen may be 0)
// aligned at the top bits, starting at base `off` of the query; bits past
// qlen or tlen are ignored.  Returns 2 when the window does not decide, else
// the outcome with *lcp set.
__device__ __forceinline__ int cmp_window(uint64_t q, uint64_t t, uint32_t qlen, uint32_t tlen, uint32_t off,
                                          uint32_t m, uint32_t *lcp) {
    const uint64_t x = q ^ t;
    const uint32_t d = x ? ((uint32_t)__clzll((long long)x) >> 1) : 32u;
    if (d < min(qlen, tlen)) {
        *lcp = off + d;
        return q < t ? CMP_LESS : CMP_GREATER;
    }
    if (tlen < qlen) {
        *lcp = off + tlen;
        return CMP_GREATER;
    }
    if (off + qlen >= m) {
        *lcp = m;
        return CMP_PREFIX;
    }
    return 2;
}

// P (bases 0-63 in q0, q1, bases 64-127 in x2, x3; length m >= 1) against a
// 32-byte suffix record (r0 = bases 0-63, r1 = bases 64-95, 96-111 and the
// position).  Sets *undecided when all 112 bases agree, m > 112 and the
// suffix has 112 bases or more; the compare then continues in the text.
__device__ __forceinline__ int cmp_record(uint64_t q0, uint64_t q1, uint64_t x2, uint64_t x3, uint32_t m, uint4 r0,
                                          uint4 r1, uint32_t n, uint32_t *lcp, bool *undecided) {
    const uint32_t klen = min(112u, n - r1.w);
    int c = cmp_window(q0, ((uint64_t)r0.y << 32) | r0.x, min(32u, m), min(32u, klen), 0u, m, lcp);
    if (c != 2) return c;
    c = cmp_window(q1, ((uint64_t)r0.w << 32) | r0.z, min(32u, m - 32u), min(32u, klen - 32u), 32u, m, lcp);
    if (c != 2) return c;
    c = cmp_window(x2, ((uint64_t)r1.y << 32) | r1.x, min(32u, m - 64u), min(32u, klen - 64u), 64u, m, lcp);
    if (c != 2) return c;
    c = cmp_window(x3 & 0xFFFFFFFF00000000ull, (uint64_t)r1.z << 32, min(16u, m - 96u), min(16u, klen - 96u), 96u,
                   m, lcp);
    if (c != 2) return c;
    *undecided = true;
    *lcp = 112;
    return CMP_PREFIX;
}

// Query P (length m >= 1, bases at base qa of the packed batch tq) against
// the suffix at p of a text of n < 2^32 bases, from the 32-aligned base below
// `start` (< m; all bases before it are known equal).
__device__ __forceinline__ int cmp_suffix_tq(const uint64_t *__restrict__ T, uint32_t n, uint32_t p,
                                             const uint64_t *__restrict__ tq, uint64_t qa, uint32_t m,
                                             uint32_t start, uint32_t *lcp) {
    uint32_t off = start & ~31u;
    const uint32_t rem = n - p;
    for (;;) {
        const uint32_t qlen = min(32u, m - off);
        const uint32_t tlen = off < rem ? min(32u, rem - off) : 0u;
        const uint64_t q = text_window(tq, qa + off);
        const uint64_t t = tlen ? text_window(T, (uint64_t)(p + off)) : 0ull;
        const int c = cmp_window(q, t, qlen, tlen, off, m, lcp);
        if (c != 2) return c;
        off += 32u;
    }
}

// The query's 32-base window at base `off` (a multiple of 32, off >= 96): base
// 96 from w3 (the query's fourth packed word), bases 128 .. 128 + 32
// tail_words - 1 from `tail` (later words its record carries, read again from
// the record when a compare gets there), the rest from the packed batch.
struct QueryWindows {
    const uint64_t *tq;
    uint64_t qa;
    uint64_t w3;
    const uint64_t *tail;
    uint32_t tail_words;
    __device__ __forceinline__ uint64_t operator()(uint32_t off) const {
        if (off == 96u) return w3;
        if (off >= 128u && ((off - 128u) >> 5) < tail_words) return __ldg(tail + ((off - 128u) >> 5));
        return text_window(tq, qa + off);
    }
};

// cmp_suffix_tq with the query's windows from qw (start >= 96).
__device__ __forceinline__ int cmp_suffix_qw(const uint64_t *__restrict__ T, uint32_t n, uint32_t p,
                                             const QueryWindows &qw, uint32_t m, uint32_t start, uint32_t *lcp) {
    uint32_t off = start & ~31u;
    const uint32_t rem = n - p;
    for (;;) {
        const uint32_t qlen = min(32u, m - off);
        const uint32_t tlen = off < rem ? min(32u, rem - off) : 0u;
        const uint64_t q = qw(off);
        const uint64_t t = tlen ? text_window(T, (uint64_t)(p + off)) : 0ull;
        const int c = cmp_window(q, t, qlen, tlen, off, m, lcp);
        if (c != 2) return c;
        off += 32u;
    }
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
    uint4 *krt;          // device, 4^kmer_k k-mer entries of 64 bytes (4 uint4) for the k-base
                         // strings x (x as a 2k-bit number): {lo, hi, pos, clamp} -- the ranks
                         // [lo, hi) of the suffixes sorting at or after x and before x + 1,
                         // lo = number of suffixes that sort before x, and the position of the
                         // suffix at the first pivot lo - 1 + (hi - lo + 1) / 2 with clamp =
                         // min(192, n - pos) -- then the first 192 bases of that suffix as six
                         // packed words; null if none
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
int build_suffix_array(sa_index *idx, cudaStream_t s);
// The same array by the paper's DC3 construction, on the GPU (dc3_gpu.cu).
int build_suffix_array_dc3(sa_index *idx, cudaStream_t s);
cudaError_t launch_build_keys(sa_index *idx, cudaStream_t s);
cudaError_t launch_build_records(sa_index *idx, cudaStream_t s);
cudaError_t launch_build_kmer(sa_index *idx, cudaStream_t s);
cudaError_t launch_copy_kmer_counts(const sa_index *idx, uint32_t *dst, cudaStream_t s);

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
    const uint64_t *tq;       // packed batch: nwords + SA_TQ_PAD_WORDS words
    const uint32_t *tv;       // per packed word: bit i set = base 32 w + i is not a base
    uint64_t nwords;          // ceil(total / 32)
    const uint64_t *q_off;    // n_q + 1 offsets
    uint64_t first;           // q_off[0]
    uint64_t total;           // q_off[n_q] - q_off[0]: query ranges past it are invalid
    const uint32_t *q_ref;    // null when n_refs == 1
    uint64_t n_q;
    uint4 *wrec;              // worklist records, 64 bytes (4 uint4) each, n_q of room
    uint32_t *wl_count;       // device: records in the worklist
    const uint4 *wrec_in;     // k-mer order: the batch's queries as records (first pass input), or null
    uint32_t *wl_in_count;    // k-mer order: records in wrec_in
    sa_result *out;
    int *pack_err;            // device flag: some query had a non-ACGT byte or bad offsets
    int *batch_dirty;         // device flag set by the packing: some byte of the batch is not a base
                              // (null: assume so).  With the flag, tv holds every mask only for a batch
                              // that is not clean; a clean batch needs (and has) none.
    int *bad_ref;             // device flag: some query named a reference id >= n_refs
    unsigned long long *counter;
    int *status;
    uint32_t smem_bytes;      // shared-memory key tables
    uint32_t threads, blocks, chunk;
    uint32_t front_probes;    // probes per query in the first pass
    bool revcomp;             // search every query's reverse complement (the batch is packed reversed)
    bool strand_bits;         // q_ref bit 31 selects each query's strand (both packings in tq)
    uint64_t rc_base;         // first base of the reverse-complement packing in tq (0: it is the only one)
    bool expire_waits;        // test hook: the bounded key-table wait gives up at once
    uint32_t trunc_cap;       // the locate cap of sa_search_locate (SA_RESULT_TRUNCATED), else ~0u
    // k-mer order (bucket.cu)
    uint64_t ktotal;          // k-mer entries of all indexes of the call
    uint32_t *bplan;          // the list's plan, kPlanWords words (see below; zeroed by the caller)
    // search + locate in one call: per 2^kLocateTileShift queries, the sum of
    // min(count, trunc_cap) of their results (zeroed by the caller), or null
    uint64_t *tile_kept;
    bool tile_sum_by_warp;    // input order: the lanes storing together mostly share a tile
};

// Queries per tile of the locate's scan (locate.cu).
constexpr uint32_t kLocateTileShift = 12;

// store_result for the search kernels; in a search + locate call it also
// adds the query's kept count min(count, cap) to its locate tile's sum, so
// the locate need not read every result to find the tile sums.
// In input order the lanes storing at the same time hold consecutive queries,
// so those sharing a tile add their counts with one atomic; in k-mer order
// each lane adds its own.
__device__ __forceinline__ void store_result_sum(const SearchLaunch &a, uint64_t q, uint64_t lo, uint64_t hi) {
    store_result(a.out, q, lo, hi, a.trunc_cap);
    if (a.tile_kept == nullptr) return;
    const uint64_t c = lo == ~0ull ? 0ull : hi - lo;
    const uint32_t k = c < (uint64_t)a.trunc_cap ? (uint32_t)c : a.trunc_cap;
    const uint64_t tile = q >> kLocateTileShift;
    unsigned long long *sum_at = reinterpret_cast<unsigned long long *>(a.tile_kept) + tile;
    if (a.tile_sum_by_warp) {
        const unsigned same = __match_any_sync(__activemask(), tile);
        const uint32_t sum = __reduce_add_sync(same, k);
        if (sum != 0u && (threadIdx.x & 31u) == (unsigned)(__ffs(same) - 1)) atomicAdd(sum_at, (unsigned long long)sum);
    } else if (k != 0u) {
        atomicAdd(sum_at, (unsigned long long)k);
    }
}
// Worklist record of a query the first pass did not finish (64 bytes):
//   {L, R, m, q}            a bracket (L, R) holding both bounds (L = -1 is
//                           0xFFFFFFFF), the length and the query's index
//   {qa.lo, qa.hi | ref << 16, w4.lo, w4.hi}  its first base in the packed
//                           batch (qa < 2^48), reference id (< 2^15) and
//                           bases 128-159
//   {w0, w1}, {w2, w3}      its first 128 bases (packed words)
cudaError_t launch_pack_batch(const SearchLaunch &L, uint64_t *tq, uint32_t *tv, cudaStream_t s);
cudaError_t launch_front(const SearchLaunch &L, cudaStream_t s);
// The batch's queries as records in k-mer order (wrec_in), the first pass's
// input in that order.
cudaError_t launch_bucketed_worklist(const SearchLaunch &L, uint4 *wrec_in, cudaStream_t s);
cudaError_t launch_search(const SearchLaunch &L, cudaStream_t s);
cudaError_t launch_search_plain(const SearchLaunch &L, cudaStream_t s);
// One thread: *dst = the call's status from its device flags (flags[1] a
// wait that ran out, flags[0] a query that is not bases, flags[3] a bad
// reference id), in that order of precedence.
cudaError_t launch_search_status(const int *flags, int *dst, cudaStream_t s);
// One thread each: fold one chunk's device flags into acc[0] (an atomic max
// of the status's precedence: 3 TIMEOUT, 2 BASE, 1 ARG, 0 OK), so that chunks
// on several streams fold into one word; then *dst = the status of acc[0], or
// SA_ERR_CAPACITY when that is SA_OK and check_overflow and acc[1] is set.
cudaError_t launch_fold_status(const int *flags, int *acc, cudaStream_t s);
cudaError_t launch_fold_final(const int *acc, bool check_overflow, int *dst, cudaStream_t s);
// One thread: *dst = SA_ERR_CAPACITY when *overflow is set and *dst is SA_OK.
cudaError_t launch_capacity_status(const int *overflow, int *dst, cudaStream_t s);
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
    bool presummed;           // partials already hold the tile sums (from the search kernels)
    int *overflow;            // optional device flag: a position fell at or beyond capacity
    const uint64_t *base_in;  // optional device value added to every offset (a chunk of a larger batch)
};
uint64_t locate_tiles(uint64_t n_q);
// Device address of the static scratch of sa_locate_noalloc on the current
// device (looked up once per device) and the number of partial sums it holds.
cudaError_t locate_static_partials(uint64_t **ptr, uint64_t *entries);
cudaError_t launch_locate(const LocateLaunch &L, cudaStream_t s);
// Copies positions [*first, *last) (clamped to capacity) of width bytes each
// from src to dst at the same indexes; dst may be host memory the device can
// address.
cudaError_t launch_copy_positions(const uint64_t *first, const uint64_t *last, const void *src, void *dst,
                                  uint32_t width, uint64_t capacity, cudaStream_t s);

}  // namespace sa
