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
// Four kernels put the batch in that order before the first pass (front.cu),
// which then reads its queries from the list they write:
//   bucket_sample_kernel   every kListSampleStride-th query's bucket -- its
//                          first k bases as a fraction of all k-mer entries
//                          of the call's indexes, in kNumBuckets equal
//                          slices, or the extra bucket of queries with no
//                          k-mer bracket -- counted;
//   bucket_plan_kernel     one warp: from those counts each bucket's region
//                          of the list (9/8 of its estimated size plus 256
//                          records), in bucket order, and after them an
//                          overflow region with room for every query;
//   bucket_scatter_kernel  per tile of queries: offsets, strand, reference,
//                          validity of every base when the packing found a
//                          non-base byte in the batch (invalid and empty
//                          queries get their results here) and bucket; each
//                          bucket's run reserved at once in its region (what
//                          does not fit goes to the overflow region), every
//                          query's 64-byte record (length, index, reference,
//                          first base in the packed batch, first 192 bases;
//                          flagged when it has a k-mer bracket to read) built
//                          in shared memory and the runs stored coalesced;
//   bucket_fill_kernel     one warp: the prefix sums of the regions' fills,
//                          by which the first pass numbers the records
//                          (region by region, then the overflow).
// The first pass and then the persistent kernel of search.cu take the queries
// in that order, so the reads in flight at any time stay in a few slices.
// Sizing the regions from a sample spares a pass over the whole batch that
// exact counts would need; the overflow region keeps the result exact
// whatever the sample missed.
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kSampleThreads = 256;
constexpr uint16_t kNoQuery = 0xFFFFu;  // invalid or empty query: no list record

struct BucketRef {
    uint64_t kbase;   // k-mer entries of the earlier indexes of the call
    uint64_t n;
    uint32_t kmer_k;  // 0: no k-mer table
};

// The query's first base in the packed batch (in the reverse-complement
// packing for the other strand), its length, its reference id (*r, the strand
// bit cleared) and whether the range and the reference id are usable.
__device__ __forceinline__ bool query_range(const SearchLaunch &a, uint64_t q, uint32_t *r, uint64_t *qa_out,
                                            uint32_t *m_out, bool *bad_range, bool *bad_ref) {
    const uint64_t qa = __ldg(a.q_off + q) - a.first, qe = __ldg(a.q_off + q + 1) - a.first;
    const bool rc = a.revcomp || (a.strand_bits && (*r & kStrandBit));
    if (a.strand_bits) *r &= ~kStrandBit;
    const bool range_ok = qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
    *bad_range = !range_ok;
    *bad_ref = range_ok && *r >= a.n_refs;
    *qa_out = range_ok ? strand_start(qa, qe, a.total, rc, a.rc_base) : qa;
    *m_out = range_ok ? (uint32_t)(qe - qa) : 0u;
    return range_ok && *r < a.n_refs;
}

// The bucket of a usable query of length m >= 1 whose first 32 bases are w0.
__device__ __forceinline__ uint16_t bucket_of(const SearchLaunch &a, const BucketRef &d, uint32_t m, uint64_t w0) {
    if (d.kmer_k != 0 && m >= d.kmer_k) {
        const uint64_t x = w0 >> (64u - 2u * d.kmer_k);
        return (uint16_t)(((d.kbase + x) * kNumBuckets) / a.ktotal);
    }
    return (uint16_t)kNumBuckets;  // no k-mer bracket: the key-table descent
}

// The query's first 32 bases from the packed batch (qa's word and the next).
__device__ __forceinline__ uint64_t first_word(const uint64_t *__restrict__ tq, uint64_t qa) {
    const uint64_t wl = qa >> 5;
    const uint32_t sh = (uint32_t)(qa & 31u) * 2u;
    return (__ldg(tq + wl) << sh) | ((__ldg(tq + wl + 1) >> 1) >> (63u - sh));
}

template <bool kSingle>
__global__ void __launch_bounds__(kSampleThreads) bucket_sample_kernel(const __grid_constant__ SearchLaunch a) {
    __shared__ uint32_t hist[kNumBuckets + 1];
    __shared__ BucketRef sref[SA_MAX_REFS];
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x) hist[i] = 0;
    for (unsigned r = threadIdx.x; r < a.n_refs; r += blockDim.x) {
        const RefDesc &d = a.refs.r[r];
        sref[r] = BucketRef{d.kbase, d.n, d.krt != nullptr ? d.kmer_k : 0u};
    }
    __syncthreads();
    const uint64_t n_s = (a.n_q + kListSampleStride - 1) / kListSampleStride;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_s; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = i * kListSampleStride;
        uint32_t r = kSingle ? 0u : __ldg(a.q_ref + q);
        uint64_t qa;
        uint32_t m;
        bool bad_range, bad_ref;
        // an estimate: the bases' validity is left to the scatter
        if (query_range(a, q, &r, &qa, &m, &bad_range, &bad_ref) && m > 0)
            atomicAdd(&hist[bucket_of(a, sref[kSingle ? 0u : r], m, first_word(a.tq, qa))], 1u);
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x)
        if (hist[i]) atomicAdd(a.bplan + kPlanSample + i, hist[i]);
}

// One warp: each bucket's region of the list and its cursor, then the
// overflow region.  A bucket sampled s times gets s * stride * 9/8 + 256
// records; the regions follow one another in bucket order.
__global__ void bucket_plan_kernel(const __grid_constant__ SearchLaunch a) {
    const unsigned lane = threadIdx.x;
    uint32_t *plan = a.bplan;
    uint32_t carry = 0;
    for (unsigned base = 0; base <= kNumBuckets; base += 32) {
        const unsigned i = base + lane;
        const uint32_t est = i <= kNumBuckets ? plan[kPlanSample + i] * kListSampleStride : 0u;
        const uint32_t v = i <= kNumBuckets ? est + est / 8u + 256u : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (i <= kNumBuckets) {
            plan[kPlanStart + i] = carry + x - v;
            plan[kPlanCursor + i] = carry + x - v;
            plan[kPlanCap + i] = v;
        }
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
    if (lane == 0) {
        plan[kPlanOvStart] = carry;
        plan[kPlanOvCursor] = carry;
    }
}

// Scatter: one CTA per tile of kScatterTile queries.  The tile's records are
// first built in shared memory in bucket order (each bucket's run of the
// tile contiguous), then copied out run by run: consecutive threads store
// consecutive 16-byte words of a run, so the stores coalesce (a record
// written straight to its slot from each lane would put the 32 lanes of a
// warp in 32 different runs).  Each bucket's run is reserved with one atomic
// on the bucket's cursor; the part past the region's end is reserved in the
// overflow region.
constexpr int kScatterThreads = 256;
constexpr int kScatterItems = 2;
constexpr uint32_t kScatterTile = (uint32_t)kScatterThreads * kScatterItems;  // 32 KB of records
constexpr size_t kScatterSmem = (size_t)kScatterTile * 64;

template <bool kSingle>
__global__ void __launch_bounds__(kScatterThreads, 5) bucket_scatter_kernel(const __grid_constant__ SearchLaunch a,
                                                                           uint4 *__restrict__ list) {
    extern __shared__ uint4 srec[];  // kScatterTile records of 4 uint4
    __shared__ uint32_t cnt[kNumBuckets + 1];
    __shared__ uint32_t off[kNumBuckets + 1];     // the run's first slot in the tile
    __shared__ uint32_t base[kNumBuckets + 1];    // its first slot in the list (in the bucket's region)
    __shared__ uint32_t inreg[kNumBuckets + 1];   // how many of the run fit the region
    __shared__ uint32_t ovbase[kNumBuckets + 1];  // the first overflow slot of the rest
    __shared__ uint16_t slot_bucket[kScatterTile];
    __shared__ BucketRef sref[SA_MAX_REFS];
    __shared__ uint32_t n_valid;
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x) cnt[i] = 0;
    for (unsigned r = threadIdx.x; r < a.n_refs; r += blockDim.x) {
        const RefDesc &d = a.refs.r[r];
        sref[r] = BucketRef{d.kbase, d.n, d.krt != nullptr ? d.kmer_k : 0u};
    }
    // a batch without a non-base byte needs no validity masks
    const bool dirty = a.batch_dirty == nullptr || *a.batch_dirty != 0;
    const uint64_t tile = (uint64_t)blockIdx.x * kScatterTile;
    uint16_t b[kScatterItems];
    uint32_t rank[kScatterItems], r[kScatterItems], m[kScatterItems];
    uint64_t qa[kScatterItems], w[kScatterItems][4];
    bool any_bad = false, any_bad_ref = false;
    __syncthreads();
    // Every item's loads are issued before the tile's bookkeeping, so that
    // their DRAM round trips overlap each other and the scans below.
#pragma unroll
    for (int it = 0; it < kScatterItems; it++) {
        const uint64_t q = tile + (uint64_t)it * kScatterThreads + threadIdx.x;
        r[it] = kSingle || q >= a.n_q ? 0u : __ldg(a.q_ref + q);
    }
#pragma unroll
    for (int it = 0; it < kScatterItems; it++) {
        const uint64_t q = tile + (uint64_t)it * kScatterThreads + threadIdx.x;
        qa[it] = 0;
        m[it] = 0;
        b[it] = kNoQuery;
        if (q < a.n_q) {
            bool bad_range, bad_ref;
            const bool ok = query_range(a, q, &r[it], &qa[it], &m[it], &bad_range, &bad_ref);
            any_bad |= bad_range;
            any_bad_ref |= bad_ref;
            b[it] = ok ? 0u : kNoQuery;  // usable so far; the bucket follows
        }
    }
#pragma unroll
    for (int it = 0; it < kScatterItems; it++) {
        const uint64_t q = tile + (uint64_t)it * kScatterThreads + threadIdx.x;
        // a query without a record reads the batch's first words (always there)
        const bool ok = b[it] != kNoQuery;
        const bool valid = load_query_head(a.tq, a.tv, ok ? qa[it] >> 5 : 0, ok ? (uint32_t)(qa[it] & 31u) : 0u,
                                           m[it], ok && m[it] > 0 && dirty, w[it]);
        if (q >= a.n_q) continue;
        if (!ok || !valid) {
            if (ok) any_bad = true;
            b[it] = kNoQuery;
            store_result_sum(a, q, ~0ull, ~0ull);
        } else if (m[it] == 0) {
            b[it] = kNoQuery;
            store_result_sum(a, q, 0, sref[kSingle ? 0u : r[it]].n);
        } else {
            b[it] = bucket_of(a, sref[kSingle ? 0u : r[it]], m[it], w[it][0]);
        }
    }
#pragma unroll
    for (int it = 0; it < kScatterItems; it++) rank[it] = b[it] != kNoQuery ? atomicAdd(&cnt[b[it]], 1u) : 0u;
    __syncthreads();
    // the tile's runs: exclusive scan of its counts (first warp), and each
    // run's place in the list, reserved with one atomic per bucket
    if (threadIdx.x < 32) {
        const unsigned lane = threadIdx.x;
        uint32_t carry = 0;
        for (unsigned s0 = 0; s0 <= kNumBuckets; s0 += 32) {
            const unsigned i = s0 + lane;
            const uint32_t v = i <= kNumBuckets ? cnt[i] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= (unsigned)o) x += y;
            }
            if (i <= kNumBuckets) off[i] = carry + x - v;
            carry += __shfl_sync(0xFFFFFFFFu, x, 31);
        }
        if (lane == 0) n_valid = carry;
    }
    for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x) {
        const uint32_t c = cnt[i];
        if (c == 0) continue;
        const uint32_t start = atomicAdd(a.bplan + kPlanCursor + i, c);
        const uint32_t end = a.bplan[kPlanStart + i] + a.bplan[kPlanCap + i];
        const uint32_t fit = start >= end ? 0u : (end - start < c ? end - start : c);
        base[i] = start;
        inreg[i] = fit;
        ovbase[i] = fit < c ? atomicAdd(a.bplan + kPlanOvCursor, c - fit) : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kScatterItems; it++) {
        if (b[it] == kNoQuery) continue;
        const uint64_t q = tile + (uint64_t)it * kScatterThreads + threadIdx.x;
        const bool entry = b[it] < kNumBuckets;
        const uint32_t slot = off[b[it]] + rank[it];
        // bases 128-191 (the first pass then reads none of a query of up to
        // 192 bases from the batch)
        uint64_t t0 = 0, t1 = 0;
        if (m[it] > 128u) {
            const uint64_t wl = qa[it] >> 5;
            const uint32_t sh = (uint32_t)(qa[it] & 31u) * 2u;
            const uint64_t x4 = __ldg(a.tq + wl + 4), x5 = __ldg(a.tq + wl + 5), x6 = __ldg(a.tq + wl + 6);
            t0 = (x4 << sh) | ((x5 >> 1) >> (63u - sh));
            t1 = (x5 << sh) | ((x6 >> 1) >> (63u - sh));
        }
        uint4 *dst = srec + 4 * slot;
        dst[0] = make_uint4(m[it], (uint32_t)q, (uint32_t)qa[it],
                            (uint32_t)(qa[it] >> 32) | (r[it] << 16) | (entry ? kListNeedsEntry : 0u));
        dst[1] = make_uint4((uint32_t)w[it][0], (uint32_t)(w[it][0] >> 32), (uint32_t)w[it][1],
                            (uint32_t)(w[it][1] >> 32));
        dst[2] = make_uint4((uint32_t)w[it][2], (uint32_t)(w[it][2] >> 32), (uint32_t)w[it][3],
                            (uint32_t)(w[it][3] >> 32));
        dst[3] = make_uint4((uint32_t)t0, (uint32_t)(t0 >> 32), (uint32_t)t1, (uint32_t)(t1 >> 32));
        slot_bucket[slot] = b[it];
    }
    __syncthreads();
    // copy the runs out, 16 bytes per thread per step
    const uint32_t words = 4u * n_valid;
    for (uint32_t c = threadIdx.x; c < words; c += kScatterThreads) {
        const uint32_t slot = c >> 2;
        const uint32_t bk = slot_bucket[slot];
        const uint32_t k = slot - off[bk];
        const uint64_t g = k < inreg[bk] ? (uint64_t)base[bk] + k : (uint64_t)ovbase[bk] + (k - inreg[bk]);
        list[4 * g + (c & 3u)] = srec[c];
    }
    const unsigned lane = threadIdx.x & 31u;
    if (__any_sync(0xFFFFFFFFu, any_bad) && lane == 0) atomicOr(a.pack_err, 1);
    if (__any_sync(0xFFFFFFFFu, any_bad_ref) && lane == 0) atomicOr(a.bad_ref, 1);
}

// One warp: the exclusive prefix sums of the regions' fills (the records
// each bucket's region received), their total, and the list's record count
// (the regions' records, then the overflow's).
__global__ void bucket_fill_kernel(const __grid_constant__ SearchLaunch a) {
    const unsigned lane = threadIdx.x;
    uint32_t *plan = a.bplan;
    uint32_t carry = 0;
    for (unsigned s0 = 0; s0 <= kNumBuckets; s0 += 32) {
        const unsigned i = s0 + lane;
        uint32_t v = 0;
        if (i <= kNumBuckets) {
            const uint32_t used = plan[kPlanCursor + i] - plan[kPlanStart + i];
            v = used < plan[kPlanCap + i] ? used : plan[kPlanCap + i];
        }
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (i <= kNumBuckets) plan[kPlanPrefix + i] = carry + x - v;
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
    if (lane == 0) {
        plan[kPlanPrefix + kNumBuckets + 1] = carry;
        *a.wl_in_count = carry + (plan[kPlanOvCursor] - plan[kPlanOvStart]);
    }
}

}  // namespace

cudaError_t launch_bucketed_worklist(const SearchLaunch &L, uint4 *wrec_in, cudaStream_t s) {
    if (L.n_q == 0) return cudaSuccess;
    const bool single = L.n_refs == 1 && L.q_ref == nullptr;
    const uint64_t n_s = (L.n_q + kListSampleStride - 1) / kListSampleStride;
    uint64_t sblocks = (n_s + kSampleThreads - 1) / kSampleThreads;
    const uint64_t scap = (uint64_t)device_sm_count() * 8;
    if (sblocks > scap) sblocks = scap;
    if (single)
        bucket_sample_kernel<true><<<(unsigned)sblocks, kSampleThreads, 0, s>>>(L);
    else
        bucket_sample_kernel<false><<<(unsigned)sblocks, kSampleThreads, 0, s>>>(L);
    bucket_plan_kernel<<<1, 32, 0, s>>>(L);
    const uint64_t stiles = (L.n_q + kScatterTile - 1) / kScatterTile;
    auto scatter = single ? bucket_scatter_kernel<true> : bucket_scatter_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    if (e != cudaSuccess) return e;
    scatter<<<(unsigned)stiles, kScatterThreads, kScatterSmem, s>>>(L, wrec_in);
    bucket_fill_kernel<<<1, 32, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace sa
