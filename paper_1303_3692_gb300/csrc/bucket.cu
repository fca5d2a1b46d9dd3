// bucket.cu -- the worklist of a batch in k-mer order, for indexes larger
// than the GPU's address-translation reach.
//
// The probes of a search are random reads into the k-mer entries and suffix
// records (Section IV's binary search, with the exact shortcuts of this
// library).  On the GB300 such reads run at about 37-40 G sectors/s while the
// reads in flight across the GPU touch no more than ~64 GB; over a 190 GB
// index, with every lane at a random place, the rate falls to ~8 G/s.  A
// batch processed in the order of its queries' first k bases keeps the reads
// in flight inside a narrow slice of the index instead (measured: 40 G/s
// within 1 GB windows of a 192 GB buffer).  Ranks follow k-mer order, so a
// query's k-mer entry and every suffix record of its bracket lie in its
// slice.
//
// Three kernels put the batch in that order before the first pass (front.cu),
// which then reads its queries from the list they write:
//   bucket_count_kernel    one thread per query: offsets, strand, reference,
//                          validity of every base (invalid and empty queries
//                          get their results here), and the query's bucket --
//                          its first k bases as a fraction of all k-mer
//                          entries of the call's indexes, in kNumBuckets
//                          equal slices, or the extra bucket of queries with
//                          no k-mer bracket; per-CTA histograms summed into a
//                          global one;
//   bucket_scan_kernel     exclusive scan of the kNumBuckets + 1 totals: each
//                          bucket's first worklist slot, and the count;
//   bucket_scatter_kernel  per tile of queries, each bucket's run reserved at
//                          once and every query's 64-byte record (length,
//                          index, reference, first base in the packed batch,
//                          first 128 bases) written at its slot, flagged when
//                          it has a k-mer bracket to read.
// The first pass and then the persistent kernel of search.cu take the queries
// in that order, so the reads in flight at any time stay in a few slices.
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kBucketThreads = 512;
constexpr int kBucketItems = 8;
constexpr uint64_t kBucketTile = (uint64_t)kBucketThreads * kBucketItems;
constexpr uint16_t kNoQuery = 0xFFFFu;  // invalid or empty query: no worklist record

struct BucketRef {
    uint64_t kbase;   // k-mer entries of the earlier indexes of the call
    uint64_t n;
    uint32_t kmer_k;  // 0: no k-mer table
};

// The query's range in the packed batch (mirrored for the other strand) and
// whether the range and the reference id are usable.
__device__ __forceinline__ bool query_range(const SearchLaunch &a, uint64_t q, uint32_t r, uint64_t *qa_out,
                                            uint32_t *m_out, bool *bad_range, bool *bad_ref) {
    uint64_t qa = __ldg(a.q_off + q) - a.first, qe = __ldg(a.q_off + q + 1) - a.first;
    const bool range_ok = qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
    *bad_range = !range_ok;
    *bad_ref = range_ok && r >= a.n_refs;
    if (range_ok && a.revcomp) {  // the reverse complement sits at the mirrored range
        const uint64_t t = a.total - qe;
        qe = a.total - qa;
        qa = t;
    }
    *qa_out = qa;
    *m_out = range_ok ? (uint32_t)(qe - qa) : 0u;
    return range_ok && r < a.n_refs;
}

template <bool kSingle>
__global__ void __launch_bounds__(kBucketThreads) bucket_count_kernel(const __grid_constant__ SearchLaunch a) {
    __shared__ uint32_t hist[kNumBuckets + 1];
    __shared__ BucketRef sref[SA_MAX_REFS];
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x) hist[i] = 0;
    for (unsigned r = threadIdx.x; r < a.n_refs; r += blockDim.x) {
        const RefDesc &d = a.refs.r[r];
        sref[r] = BucketRef{d.kbase, d.n, d.krt != nullptr ? d.kmer_k : 0u};
    }
    __syncthreads();
    bool any_bad = false, any_bad_ref = false;
    const uint64_t tile = (uint64_t)blockIdx.x * kBucketTile;
#pragma unroll 1
    for (int it = 0; it < kBucketItems; it++) {
        const uint64_t q = tile + (uint64_t)it * kBucketThreads + threadIdx.x;
        if (q >= a.n_q) break;
        const uint32_t r = kSingle ? 0u : __ldg(a.q_ref + q);
        uint64_t qa;
        uint32_t m;
        bool bad_range, bad_ref;
        bool ok = query_range(a, q, r, &qa, &m, &bad_range, &bad_ref);
        any_bad |= bad_range;
        any_bad_ref |= bad_ref;
        uint64_t w[4];
        if (!load_query_head(a.tq, a.tv, ok ? (qa >> 5) : 0, (uint32_t)(qa & 31u), m, ok && m > 0, w)) {
            ok = false;
            any_bad = true;
        }
        uint16_t b = kNoQuery;
        if (!ok) {
            store_result(a.out, q, ~0ull, ~0ull, a.trunc_cap);
        } else {
            const BucketRef d = sref[kSingle ? 0u : r];
            if (m == 0) {
                store_result(a.out, q, 0, d.n, a.trunc_cap);
            } else if (d.kmer_k != 0 && m >= d.kmer_k) {
                const uint64_t x = w[0] >> (64u - 2u * d.kmer_k);
                b = (uint16_t)(((d.kbase + x) * kNumBuckets) / a.ktotal);
            } else {
                b = (uint16_t)kNumBuckets;  // no k-mer bracket: the key-table descent
            }
        }
        if (b != kNoQuery) atomicAdd(&hist[b], 1u);
        a.qbucket[q] = b;
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x)
        if (hist[i]) atomicAdd(a.bhist + i, hist[i]);
    if (any_bad) atomicOr(a.pack_err, 1);
    if (any_bad_ref) atomicOr(a.bad_ref, 1);
}

// One warp: bcursor[b] = the totals of the buckets before b; the worklist
// count is their sum.
__global__ void bucket_scan_kernel(const __grid_constant__ SearchLaunch a) {
    const unsigned lane = threadIdx.x;
    uint32_t carry = 0;
    for (unsigned base = 0; base <= kNumBuckets; base += 32) {
        const unsigned i = base + lane;
        const uint32_t v = i <= kNumBuckets ? a.bhist[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (i <= kNumBuckets) a.bcursor[i] = carry + x - v;
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
    if (lane == 0) *a.wl_in_count = carry;
}

template <bool kSingle>
__global__ void __launch_bounds__(kBucketThreads) bucket_scatter_kernel(const __grid_constant__ SearchLaunch a,
                                                                       uint4 *__restrict__ list) {
    __shared__ uint32_t cnt[kNumBuckets + 1];
    __shared__ uint32_t base[kNumBuckets + 1];
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const uint64_t tile = (uint64_t)blockIdx.x * kBucketTile;
    uint16_t b[kBucketItems];
    uint32_t rank[kBucketItems];
#pragma unroll
    for (int it = 0; it < kBucketItems; it++) {
        const uint64_t q = tile + (uint64_t)it * kBucketThreads + threadIdx.x;
        b[it] = q < a.n_q ? a.qbucket[q] : kNoQuery;
        rank[it] = b[it] != kNoQuery ? atomicAdd(&cnt[b[it]], 1u) : 0u;
    }
    __syncthreads();
    // each bucket's run of this tile, reserved with one atomic
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x)
        base[i] = cnt[i] ? atomicAdd(a.bcursor + i, cnt[i]) : 0u;
    __syncthreads();
#pragma unroll 1
    for (int it = 0; it < kBucketItems; it++) {
        if (b[it] == kNoQuery) continue;
        const uint64_t q = tile + (uint64_t)it * kBucketThreads + threadIdx.x;
        const uint32_t r = kSingle ? 0u : __ldg(a.q_ref + q);
        uint64_t qa;
        uint32_t m;
        bool bad_range, bad_ref;
        query_range(a, q, r, &qa, &m, &bad_range, &bad_ref);
        uint64_t w[4];
        load_query_head(a.tq, a.tv, qa >> 5, (uint32_t)(qa & 31u), m, false, w);
        const bool entry = b[it] < kNumBuckets;
        const uint32_t n = (uint32_t)a.refs.r[kSingle ? 0u : r].n;
        uint4 *dst = list + 4 * (size_t)(base[b[it]] + rank[it]);
        // bracket (-1, n) for a query without a k-mer bracket; an entry
        // record's bracket comes from its k-mer entry
        dst[0] = make_uint4(0xFFFFFFFFu, entry ? 0u : n, m, (uint32_t)q);
        dst[1] = make_uint4(r, entry ? kRecNeedsEntry : 0u, (uint32_t)qa, (uint32_t)(qa >> 32));
        dst[2] = make_uint4((uint32_t)w[0], (uint32_t)(w[0] >> 32), (uint32_t)w[1], (uint32_t)(w[1] >> 32));
        dst[3] = make_uint4((uint32_t)w[2], (uint32_t)(w[2] >> 32), (uint32_t)w[3], (uint32_t)(w[3] >> 32));
    }
}

}  // namespace

cudaError_t launch_bucketed_worklist(const SearchLaunch &L, uint4 *wrec_in, cudaStream_t s) {
    if (L.n_q == 0) return cudaSuccess;
    const bool single = L.n_refs == 1 && L.q_ref == nullptr;
    const uint64_t tiles = (L.n_q + kBucketTile - 1) / kBucketTile;
    if (single)
        bucket_count_kernel<true><<<(unsigned)tiles, kBucketThreads, 0, s>>>(L);
    else
        bucket_count_kernel<false><<<(unsigned)tiles, kBucketThreads, 0, s>>>(L);
    bucket_scan_kernel<<<1, 32, 0, s>>>(L);
    if (single)
        bucket_scatter_kernel<true><<<(unsigned)tiles, kBucketThreads, 0, s>>>(L, wrec_in);
    else
        bucket_scatter_kernel<false><<<(unsigned)tiles, kBucketThreads, 0, s>>>(L, wrec_in);
    return cudaGetLastError();
}

}  // namespace sa
