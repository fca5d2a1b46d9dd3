// front.cu -- first pass of the search (Section IV): one thread per query.
//
// Most queries of a batch are decided by their k-mer bracket and one or two
// probes, so the first pass runs them straight through, one query per thread
// and no shared state:
//   * in input order the query's first 128 bases come from the packed batch
//     (five words of a 38-byte-per-100-bases array that the packing kernel
//     has just written) and, when the packing found a non-base byte in the
//     batch, its validity from the per-base masks; in k-mer order its record
//     in the list (bucket.cu) holds its first 192 bases, already checked;
//   * for m >= k one aligned 64-byte read of the k-mer entry of its first k
//     bases x gives the bracket (lo - 1, hi) of the suffixes that sort
//     between x and x + 1 and the suffix at the bracket's first pivot (its
//     position and first 192 bases), so the bracket and the first probe cost
//     one access;
//   * further probes of the lockstep lower/upper bound, one 32-byte suffix
//     record each, as in the persistent kernel, up to `front_probes` probes
//     in all.
// A query still undecided after that (a bracket wider than the probes could
// resolve, a query shorter than k, an index without a k-mer table) is
// appended to a worklist -- a 64-byte record holding a bracket of both
// bounds, its length, index, reference, first base in the packed batch and
// first 160 bases -- which the persistent kernel of search.cu then finishes.
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kFrontThreads = 256;

struct FrontDesc {
    const uint64_t *text;
    const uint4 *rec;
    const uint4 *krt;
    uint32_t n;
    uint32_t kmer_k;
};

// P (bases 0-127 in w, the rest from qw; length m >= 1) against the pivot of
// a k-mer entry: its first 192 bases in e (clamp of them exist), then the
// text from position pos + 192 when all 192 tie.
__device__ __forceinline__ int cmp_entry(const uint64_t w[4], uint32_t m, const uint64_t e[6], uint32_t pos,
                                         uint32_t clamp, uint32_t n, const uint64_t *__restrict__ T,
                                         const QueryWindows &qw, uint32_t *lcp) {
#pragma unroll
    for (int j = 0; j < 6; j++) {
        const uint32_t off = 32u * j;
        const uint32_t qlen = min(32u, m - off);
        const uint32_t tlen = clamp > off ? min(32u, clamp - off) : 0u;
        const uint64_t q = j < 4 ? w[j] : qw(off);
        const int c = cmp_window(q, e[j], qlen, tlen, off, m, lcp);
        if (c != 2) return c;
    }
    return cmp_suffix_qw(T, n, pos, qw, m, 192u, lcp);
}

// The list slot of the j-th record of the k-mer-ordered list: region by
// region (in the largest bucket b whose regions before it hold at most j
// records), then the overflow region.  prefix: the exclusive sums of the
// regions' fills (kNumBuckets + 2 entries, the last their total); start: each
// region's first slot.
__device__ __forceinline__ uint32_t list_slot(const uint32_t *prefix, const uint32_t *start, uint32_t ov_start,
                                              uint32_t j) {
    const uint32_t in_regions = prefix[kNumBuckets + 1];
    if (j >= in_regions) return ov_start + (j - in_regions);
    uint32_t lo = 0, hi = kNumBuckets + 1;  // prefix[lo] <= j < prefix[hi]
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (prefix[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    return start[lo] + (j - prefix[lo]);
}

// kFromList: the queries come from the k-mer-ordered list of bucket.cu (one
// 64-byte record each: length, index, reference, first base in the packed
// batch and first 192 bases, already checked) instead of the batch's offsets.
template <bool kSingle, bool kFromList>
__global__ void __launch_bounds__(kFrontThreads, 4) front_kernel(const __grid_constant__ SearchLaunch a) {
    __shared__ FrontDesc sdesc[SA_MAX_REFS];
    __shared__ uint4 s_stage[kFrontThreads / 32][32][4];  // worklist records staged per warp
    __shared__ uint32_t s_lprefix[kNumBuckets + 2];        // the list's numbering (list input)
    __shared__ uint32_t s_lstart[kNumBuckets + 1];
    for (unsigned r = threadIdx.x; r < a.n_refs; r += blockDim.x) {
        const RefDesc &d = a.refs.r[r];
        sdesc[r] = FrontDesc{d.text, d.rec, d.krt, (uint32_t)d.n, d.kmer_k};
    }
    if (kFromList) {
        for (unsigned i = threadIdx.x; i < kNumBuckets + 2; i += blockDim.x) s_lprefix[i] = a.bplan[kPlanPrefix + i];
        for (unsigned i = threadIdx.x; i <= kNumBuckets; i += blockDim.x) s_lstart[i] = a.bplan[kPlanStart + i];
    }
    const uint32_t ov_start = kFromList ? a.bplan[kPlanOvStart] : 0u;
    __syncthreads();

    const unsigned lane = threadIdx.x & 31u;
    const unsigned wib = threadIdx.x >> 5;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    uint32_t staged = 0;  // warp-uniform: records in s_stage[wib]
    // Moves the warp's staged records to the worklist (one atomic).
    auto flush = [&](uint32_t cnt) {
        if (cnt == 0u) return;
        uint32_t at = 0;
        if (lane == 0) at = atomicAdd(a.wl_count, cnt);
        at = __shfl_sync(0xFFFFFFFFu, at, 0);
        if (lane < cnt) {
            uint4 *dst = a.wrec + 4 * (size_t)(at + lane);
#pragma unroll
            for (int j = 0; j < 4; j++) dst[j] = s_stage[wib][lane][j];
        }
        __syncwarp();
    };
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t warp_first = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    const uint64_t *__restrict__ tq = a.tq;
    bool any_bad = false, any_bad_ref = false;

    const uint64_t n_items = kFromList ? (uint64_t)*a.wl_in_count : a.n_q;
    // a batch without a non-base byte needs no per-query validity check
    const bool dirty = a.batch_dirty == nullptr || *a.batch_dirty != 0;
    // Offsets and reference of this lane's next query, read one query ahead.
    uint64_t nqa = 0, nqe = 0;
    uint32_t nr = 0;
    if (!kFromList && warp_first + lane < a.n_q) {
        nqa = __ldg(a.q_off + warp_first + lane);
        nqe = __ldg(a.q_off + warp_first + lane + 1);
        if (!kSingle) nr = __ldg(a.q_ref + warp_first + lane);
    }

    for (uint64_t base = warp_first; base < n_items; base += stride) {
        const bool live = base + lane < n_items;
        uint64_t q, qa;
        uint32_t r, m;
        bool ok, entry = true;
        uint64_t w[4];
        uint32_t lslot = 0;  // the record's slot in the list (list input)
        if (kFromList) {
            uint4 c0, c1, c2, c3;
            if (live) lslot = list_slot(s_lprefix, s_lstart, ov_start, (uint32_t)(base + lane));
            const uint4 *src = a.wrec_in + 4 * (size_t)lslot;
            ldg32_if(live, src, &c0, &c1);
            ldg32_if(live, src + 2, &c2, &c3);
            m = c0.x;
            q = c0.y;
            qa = ((uint64_t)(c0.w & 0xFFFFu) << 32) | c0.z;
            r = (c0.w >> 16) & 0x7FFFu;
            entry = (c0.w & kListNeedsEntry) != 0u;
            w[0] = ((uint64_t)c1.y << 32) | c1.x;
            w[1] = ((uint64_t)c1.w << 32) | c1.z;
            w[2] = ((uint64_t)c2.y << 32) | c2.x;
            w[3] = ((uint64_t)c2.w << 32) | c2.z;
            ok = live;
        } else {
            q = base + lane;
            qa = nqa - a.first;
            const uint64_t qe = nqe - a.first;
            r = nr;
            if (base + stride + lane < a.n_q) {
                nqa = __ldg(a.q_off + base + stride + lane);
                nqe = __ldg(a.q_off + base + stride + lane + 1);
                if (!kSingle) nr = __ldg(a.q_ref + base + stride + lane);
            }
            const bool rc = a.revcomp || (a.strand_bits && (r & kStrandBit));
            if (a.strand_bits) r &= ~kStrandBit;
            const bool range_ok = live && qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
            if (live && !range_ok) any_bad = true;
            ok = range_ok && r < a.n_refs;
            if (range_ok && r >= a.n_refs) any_bad_ref = true;
            m = ok ? (uint32_t)(qe - qa) : 0u;
            if (range_ok) qa = strand_start(qa, qe, a.total, rc, a.rc_base);

            // First 128 bases and the validity of every base of the query.
            if (!load_query_head(tq, a.tv, ok ? (qa >> 5) : 0, (uint32_t)(qa & 31u), m, ok && m > 0 && dirty, w)) {
                ok = false;
                any_bad = true;
            }
        }

        FrontDesc d = sdesc[0];
        if (!kSingle && ok) d = sdesc[r];
        // Bracket and first pivot: the k-mer entry for m >= k, else the whole array.
        const uint32_t kk = d.kmer_k;
        const bool look = ok && entry && m > 0 && d.krt != nullptr && m >= kk;
        const uint64_t x = look ? (w[0] >> (64u - 2u * kk)) : 0ull;
        uint4 h, e01, e23, e45;
        ldg32_if(look, d.krt + 4 * x, &h, &e01);
        ldg32_if(look, d.krt + 4 * x + 2, &e23, &e45);
        uint32_t L = look ? h.x - 1u : 0xFFFFFFFFu;  // 0xFFFFFFFF stands for -1
        uint32_t R = look ? h.y : d.n;

        bool done = !live || !ok || m == 0 || (look && R - L <= 1u);
        if (live && !ok) store_result_sum(a, q, ~0ull, ~0ull);
        if (live && ok && m == 0) store_result_sum(a, q, 0, d.n);
        if (live && ok && m > 0 && look && R - L <= 1u) store_result_sum(a, q, R, R);

        uint32_t lcpL = 0, lcpR = 0, HL = 0, HR = 0, hlcpL = 0, hlcpR = 0, lo = 0, phase = 0;
        bool go = !done && look;
        // in list order, bases 128-191 are the record's last 16 bytes (read
        // again when a compare gets there: an L1 or L2 hit)
        const QueryWindows qw{tq, qa, w[3],
                              kFromList ? reinterpret_cast<const uint64_t *>(a.wrec_in + 4 * (size_t)lslot + 3)
                                        : nullptr,
                              kFromList ? 2u : 0u};
        // One compare's outcome c at pivot M with common prefix l.
        auto step = [&](int c, uint32_t M, uint32_t l) {
            if (c == CMP_PREFIX && phase == 0) {
                HL = M;
                hlcpL = m;
                HR = R;
                hlcpR = lcpR;
                R = M;
                lcpR = m;
                phase = 1;
            } else if (c == CMP_LESS || (c == CMP_PREFIX && phase == 1)) {
                R = M;
                lcpR = l;
            } else {
                L = M;
                lcpL = l;
            }
            if (R - L <= 1u) {
                if (phase == 1) {
                    lo = R;
                    L = HL;
                    R = HR;
                    lcpL = hlcpL;
                    lcpR = hlcpR;
                    phase = 2;
                }
                if (R - L <= 1u) {
                    store_result_sum(a, q, phase == 0 ? R : lo, R);
                    done = true;
                    go = false;
                }
            }
        };
        if (go) {  // the first probe: the entry's pivot
            const uint64_t e[6] = {((uint64_t)e01.y << 32) | e01.x, ((uint64_t)e01.w << 32) | e01.z,
                                   ((uint64_t)e23.y << 32) | e23.x, ((uint64_t)e23.w << 32) | e23.z,
                                   ((uint64_t)e45.y << 32) | e45.x, ((uint64_t)e45.w << 32) | e45.z};
            uint32_t l;
            const int c = cmp_entry(w, m, e, h.z, h.w, d.n, d.text, qw, &l);
            step(c, L + ((R - L) >> 1), l);
        }
        // Further probes, one suffix record each; queries without a k-mer
        // bracket go straight to the worklist (the persistent kernel descends
        // the shared-memory key table first).
        for (uint32_t p = 1; p < a.front_probes && __any_sync(0xFFFFFFFFu, go); p++) {
            const uint32_t M = L + ((R - L) >> 1);
            uint4 r0, r1;
            ldg32_if(go, d.rec + 2 * (size_t)M, &r0, &r1);
            if (go) {
                uint32_t l;
                bool und = false;
                int c = cmp_record(w[0], w[1], w[2], w[3], m, r0, r1, d.n, &l, &und);
                if (und) c = cmp_suffix_qw(d.text, d.n, r1.w, qw, m, max(112u, min(lcpL, lcpR)), &l);
                step(c, M, l);
            }
        }

        // The rest goes to the worklist with one bracket of both bounds:
        // phase 0 (L, R); phase 1 (L, HR) (lo in (L, M], hi in [M, HR));
        // phase 2 (lo - 1, R) (lo known, hi in (L, R) with L >= lo).  Records
        // are staged per warp in shared memory and flushed 32 at a time, so
        // the global count takes one atomic per 32 records.
        const bool rest = live && !done;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, rest);
        if (bal != 0u) {
            const uint32_t n_new = (uint32_t)__popc(bal);
            if (staged + n_new > 32u) {
                flush(staged);
                staged = 0;
            }
            if (rest) {
                const uint32_t slot = staged + __popc(bal & lanemask_lt);
                s_stage[wib][slot][0] = make_uint4(phase == 2 ? lo - 1u : L, phase == 1 ? HR : R, m, (uint32_t)q);
                const uint64_t w4 = m > 128u ? qw(128u) : 0ull;  // bases 128-159 for the persistent pass
                s_stage[wib][slot][1] =
                    make_uint4((uint32_t)qa, (uint32_t)(qa >> 32) | (r << 16), (uint32_t)w4, (uint32_t)(w4 >> 32));
                s_stage[wib][slot][2] =
                    make_uint4((uint32_t)w[0], (uint32_t)(w[0] >> 32), (uint32_t)w[1], (uint32_t)(w[1] >> 32));
                s_stage[wib][slot][3] =
                    make_uint4((uint32_t)w[2], (uint32_t)(w[2] >> 32), (uint32_t)w[3], (uint32_t)(w[3] >> 32));
            }
            staged += n_new;
            __syncwarp();
        }
    }
    flush(staged);
    if (!kFromList) {
        if (__any_sync(0xFFFFFFFFu, any_bad) && lane == 0) atomicOr(a.pack_err, 1);
        if (__any_sync(0xFFFFFFFFu, any_bad_ref) && lane == 0) atomicOr(a.bad_ref, 1);
    }
}

}  // namespace

cudaError_t launch_front(const SearchLaunch &L, cudaStream_t s) {
    if (L.n_q == 0) return cudaSuccess;
    const bool single = L.n_refs == 1 && L.q_ref == nullptr;
    const bool list = L.wrec_in != nullptr;
    static int per_sm[4][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    auto kernel = single ? (list ? front_kernel<true, true> : front_kernel<true, false>)
                         : (list ? front_kernel<false, true> : front_kernel<false, false>);
    int &bps = per_sm[(single ? 1 : 0) + (list ? 2 : 0)][dev];
    if (bps == 0) {
        int b = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kFrontThreads, 0);
        if (e != cudaSuccess) return e;
        bps = b > 0 ? b : 1;
    }
    const uint64_t warps = (L.n_q + 31) / 32;
    const uint64_t cap = (uint64_t)device_sm_count() * bps;
    uint64_t blocks = (warps + kFrontThreads / 32 - 1) / (kFrontThreads / 32);
    if (blocks > cap) blocks = cap;
    kernel<<<(unsigned)blocks, kFrontThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace sa
