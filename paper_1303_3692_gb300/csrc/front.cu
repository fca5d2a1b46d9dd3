// front.cu -- first pass of the search (Section IV): one thread per query.
//
// Most queries of a batch are decided by their k-mer bracket and one or two
// probes, so the first pass runs them straight through, one query per thread
// and no shared state:
//   * the query's first 128 bases come from the packed batch (five words of a
//     38-byte-per-100-bases array that the packing kernel has just written,
//     so they are L2 hits) and its validity from the batch's per-base masks;
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
// first 128 bases -- which the persistent kernel of search.cu then finishes.
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

__device__ __forceinline__ void write_result(sa_result *out, uint64_t q, uint64_t lo, uint64_t hi) {
    sa_result r;
    r.lo = lo;
    r.hi = hi;
    r.count = (lo == ~0ull) ? ~0ull : hi - lo;
    out[q] = r;
}

// Bits [lo, hi) of a 32-bit mask (0 <= lo <= hi <= 32).
__device__ __forceinline__ uint32_t bit_range(uint32_t lo, uint32_t hi) {
    const uint32_t upto = hi >= 32u ? 0xFFFFFFFFu : ((1u << hi) - 1u);
    return upto & ~((1u << lo) - 1u);
}

// P (bases 0-127 in w, the rest at base qa of the packed batch; length m >=
// 1) against the pivot of a k-mer entry: its first 192 bases in e (clamp of
// them exist), then the text from position pos + 192 when all 192 tie.
__device__ __forceinline__ int cmp_entry(const uint64_t w[4], uint32_t m, const uint64_t e[6], uint32_t pos,
                                         uint32_t clamp, uint32_t n, const uint64_t *__restrict__ T,
                                         const uint64_t *__restrict__ tq, uint64_t qa, uint32_t *lcp) {
#pragma unroll
    for (int j = 0; j < 6; j++) {
        const uint32_t off = 32u * j;
        const uint32_t qlen = min(32u, m - off);
        const uint32_t tlen = clamp > off ? min(32u, clamp - off) : 0u;
        const uint64_t q = j < 4 ? w[j] : text_window(tq, qa + off);
        const int c = cmp_window(q, e[j], qlen, tlen, off, m, lcp);
        if (c != 2) return c;
    }
    return cmp_suffix_tq(T, n, pos, tq, qa, m, 192u, lcp);
}

template <bool kSingle>
__global__ void __launch_bounds__(kFrontThreads, 4) front_kernel(const __grid_constant__ SearchLaunch a) {
    __shared__ FrontDesc sdesc[SA_MAX_REFS];
    __shared__ uint4 s_stage[kFrontThreads / 32][32][4];  // worklist records staged per warp
    for (unsigned r = threadIdx.x; r < a.n_refs; r += blockDim.x) {
        const RefDesc &d = a.refs.r[r];
        sdesc[r] = FrontDesc{d.text, d.rec, d.krt, (uint32_t)d.n, d.kmer_k};
    }
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

    // Offsets and reference of this lane's next query, read one query ahead.
    uint64_t nqa = 0, nqe = 0;
    uint32_t nr = 0;
    if (warp_first + lane < a.n_q) {
        nqa = __ldg(a.q_off + warp_first + lane);
        nqe = __ldg(a.q_off + warp_first + lane + 1);
        if (!kSingle) nr = __ldg(a.q_ref + warp_first + lane);
    }

    for (uint64_t base = warp_first; base < a.n_q; base += stride) {
        const uint64_t q = base + lane;
        const bool live = q < a.n_q;
        uint64_t qa = nqa - a.first, qe = nqe - a.first;
        const uint32_t r = nr;
        if (base + stride + lane < a.n_q) {
            nqa = __ldg(a.q_off + base + stride + lane);
            nqe = __ldg(a.q_off + base + stride + lane + 1);
            if (!kSingle) nr = __ldg(a.q_ref + base + stride + lane);
        }
        const bool range_ok = live && qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
        if (live && !range_ok) any_bad = true;
        if (range_ok && a.revcomp) {  // the reverse complement sits at the mirrored range
            const uint64_t t = a.total - qe;
            qe = a.total - qa;
            qa = t;
        }
        bool ok = range_ok && r < a.n_refs;
        if (range_ok && r >= a.n_refs) any_bad_ref = true;
        const uint32_t m = ok ? (uint32_t)(qe - qa) : 0u;

        // First 128 bases and the validity of every base of the query.
        const uint64_t w_lo = ok ? (qa >> 5) : 0;
        const uint32_t sh = (uint32_t)(qa & 31u) * 2u;
        uint64_t t[5];
        uint32_t v[5];
#pragma unroll
        for (int i = 0; i < 5; i++) {
            t[i] = __ldg(tq + w_lo + i);
            v[i] = __ldg(a.tv + w_lo + i);
        }
        uint64_t w[4];
#pragma unroll
        for (int j = 0; j < 4; j++) w[j] = (t[j] << sh) | ((t[j + 1] >> 1) >> (63u - sh));
        if (ok && m > 0) {
            const uint32_t b0 = (uint32_t)(qa & 31u);  // the query's first bit in word w_lo
            uint32_t badbits = 0;
#pragma unroll
            for (int i = 0; i < 5; i++) {
                const uint32_t lo = i == 0 ? b0 : 0u;
                const uint64_t end = (uint64_t)b0 + m;  // one past the query's last bit, from word w_lo
                const uint64_t wend = 32ull * (i + 1);
                const uint32_t hi = end >= wend ? 32u : (end > 32ull * i ? (uint32_t)(end - 32ull * i) : 0u);
                if (hi > lo) badbits |= v[i] & bit_range(lo, hi);
            }
            for (uint64_t i = 5; 32ull * i < (uint64_t)b0 + m; i++) {  // queries longer than 128 bases
                const uint64_t end = (uint64_t)b0 + m;
                const uint32_t hi = end >= 32ull * (i + 1) ? 32u : (uint32_t)(end - 32ull * i);
                badbits |= __ldg(a.tv + w_lo + i) & bit_range(0, hi);
            }
            if (badbits) {
                ok = false;
                any_bad = true;
            }
        }

        FrontDesc d = sdesc[0];
        if (!kSingle && ok) d = sdesc[r];
        // Bracket and first pivot: the k-mer entry for m >= k, else the whole array.
        const uint32_t kk = d.kmer_k;
        const bool look = ok && m > 0 && d.krt != nullptr && m >= kk;
        const uint64_t x = look ? (w[0] >> (64u - 2u * kk)) : 0ull;
        uint4 h, e01, e23, e45;
        ldg32_if(look, d.krt + 4 * x, &h, &e01);
        ldg32_if(look, d.krt + 4 * x + 2, &e23, &e45);
        uint32_t L = look ? h.x - 1u : 0xFFFFFFFFu;  // 0xFFFFFFFF stands for -1
        uint32_t R = look ? h.y : d.n;

        bool done = !live || !ok || m == 0 || (look && R - L <= 1u);
        if (live && !ok) write_result(a.out, q, ~0ull, ~0ull);
        if (live && ok && m == 0) write_result(a.out, q, 0, d.n);
        if (live && ok && m > 0 && look && R - L <= 1u) write_result(a.out, q, R, R);

        uint32_t lcpL = 0, lcpR = 0, HL = 0, HR = 0, hlcpL = 0, hlcpR = 0, lo = 0, phase = 0;
        bool go = !done && look;
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
                    write_result(a.out, q, phase == 0 ? R : lo, R);
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
            const int c = cmp_entry(w, m, e, h.z, h.w, d.n, d.text, tq, qa, &l);
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
                if (und) c = cmp_suffix_tq(d.text, d.n, r1.w, tq, qa, m, max(112u, min(lcpL, lcpR)), &l);
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
                s_stage[wib][slot][1] = make_uint4(r, 0u, (uint32_t)qa, (uint32_t)(qa >> 32));
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
    if (__any_sync(0xFFFFFFFFu, any_bad) && lane == 0) atomicOr(a.pack_err, 1);
    if (__any_sync(0xFFFFFFFFu, any_bad_ref) && lane == 0) atomicOr(a.bad_ref, 1);
}

}  // namespace

cudaError_t launch_front(const SearchLaunch &L, cudaStream_t s) {
    if (L.n_q == 0) return cudaSuccess;
    const bool single = L.n_refs == 1 && L.q_ref == nullptr;
    static int per_sm[2][64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int &bps = per_sm[single ? 1 : 0][dev];
    if (bps == 0) {
        int b = 0;
        const cudaError_t e = single ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, front_kernel<true>,
                                                                                    kFrontThreads, 0)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, front_kernel<false>,
                                                                                    kFrontThreads, 0);
        if (e != cudaSuccess) return e;
        bps = b > 0 ? b : 1;
    }
    const uint64_t warps = (L.n_q + 31) / 32;
    const uint64_t cap = (uint64_t)device_sm_count() * bps;
    uint64_t blocks = (warps + kFrontThreads / 32 - 1) / (kFrontThreads / 32);
    if (blocks > cap) blocks = cap;
    if (single)
        front_kernel<true><<<(unsigned)blocks, kFrontThreads, 0, s>>>(L);
    else
        front_kernel<false><<<(unsigned)blocks, kFrontThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace sa
