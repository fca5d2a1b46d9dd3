// search.cu -- the suffix-array interval of every query (Section IV).
//
// search_kernel (second pass of the product path).  Persistent CTAs, one
//   query of the first pass's worklist per lane (the queries front_kernel
//   did not finish: wide brackets, queries shorter than k, indexes without a
//   k-mer table).
//   * Each CTA first copies every index's sampled-key table into shared
//     memory with bulk asynchronous copies (cp.async.bulk, completion on an
//     mbarrier with a bounded wait).  The table holds the first 64 bases of
//     the suffixes at ranks floor((2p+1) n / 2^(l+1)) in level order, so
//     walking it is the first d levels of the binary search, in shared
//     memory instead of HBM (the paper's tiles, Section IV and V, recast).
//   * The lower and upper bound move in lockstep while they share an
//     interval (one probe serves both, the three cases of Section IV) and
//     split when a pivot's suffix has the query as a prefix.
//   * A compare starts at min(lcp(P, S_L), lcp(P, S_R)): every suffix between
//     the bounds shares that prefix with P, so it need not be re-read.  Bases
//     are compared 32 at a time (an XOR and a count of leading zeros).
//   * Each lane takes a new query as soon as its own finishes; warps take
//     chunks of queries from one global counter.  The 32 lanes of a warp
//     therefore keep 32 independent random probes in flight per load
//     instruction.
//
// search_plain_kernel (comparison point).  The paper's direct scheme
//   (Section IV): one thread per query, two independent binary searches over
//   the whole suffix array (lower and upper bound of the query), bases
//   compared one at a time against the text.
#include <type_traits>

#include "sa_internal.cuh"

namespace sa {

namespace {

struct SmemDesc {
    const uint64_t *text;
    const void *sa;
    const uint4 *rec;
    const uint4 *krt;
    uint64_t n;
    uint32_t off;
    uint32_t depth;
    uint32_t kmer_k;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity, giving up after limit_ns (a
// zero limit gives up at once without looking: the error-path test hook).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (limit_ns == 0) return false;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

__host__ __device__ __forceinline__ uint32_t table_key_bytes(uint32_t d) { return 16u << d; }
__host__ __device__ __forceinline__ uint32_t table_len_bytes(uint32_t d) { return d >= 4 ? (1u << d) : 16u; }

// P's first 64 bases (q0, q1) against a 64-base key of length klen.  Sets
// *undecided when both agree on 64 bases, m > 64 and the key has 64 bases.
__device__ __forceinline__ int cmp_key(uint64_t q0, uint64_t q1, uint32_t m, uint4 kv, uint32_t klen,
                                       uint32_t *lcp, bool *undecided) {
    const uint64_t k0 = ((uint64_t)kv.y << 32) | kv.x;
    const uint64_t k1 = ((uint64_t)kv.w << 32) | kv.z;
    uint32_t qlen = min(32u, m), tlen = min(32u, klen);
    uint64_t x = q0 ^ k0;
    uint32_t d = x ? ((uint32_t)__clzll((long long)x) >> 1) : 32u;
    if (d < min(qlen, tlen)) {
        *lcp = d;
        return q0 < k0 ? CMP_LESS : CMP_GREATER;
    }
    if (tlen < qlen) {
        *lcp = tlen;
        return CMP_GREATER;
    }
    if (m <= 32) {
        *lcp = m;
        return CMP_PREFIX;
    }
    qlen = min(32u, m - 32u);
    tlen = klen > 32u ? min(32u, klen - 32u) : 0u;
    x = q1 ^ k1;
    d = x ? ((uint32_t)__clzll((long long)x) >> 1) : 32u;
    if (d < min(qlen, tlen)) {
        *lcp = 32u + d;
        return q1 < k1 ? CMP_LESS : CMP_GREATER;
    }
    if (tlen < qlen) {
        *lcp = 32u + tlen;
        return CMP_GREATER;
    }
    if (m <= 64) {
        *lcp = m;
        return CMP_PREFIX;
    }
    *undecided = true;
    *lcp = 64;
    return CMP_PREFIX;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s for the key-table copy

// The search of one query is a sequence of steps, one per loop iteration of
// its lane, and every step that touches device memory issues one round of
// independent loads, so that the 32 lanes of a warp wait for one round per
// iteration (a lane starting a query never holds up the lanes that probe):
//   init      read the query's worklist record (bracket, length, index,
//             first base in the packed batch, reference, first 64 bases); a
//             query with a k-mer bracket probes from it, any other descends
//             the key table first;
//   descent   compare with the key of level-order node k in shared memory
//             (k = 0 once the table's depth is passed or the bounds split);
//   deep      load the suffix record of rank M = L + (R - L)/2 (32 bytes: 112
//             bases and SA[M]) -- with query bases 64-127 from the worklist
//             record in the same round -- and compare; only when all 112
//             bases tie does the compare continue in the packed text.
// Ranks are 32-bit modular: L = 0xFFFFFFFF stands for -1, and since every
// rank is in [-1, n] with n < 2^32 - 1, R - L and L + (R - L)/2 are exact.
// phase 0: both bounds share (L, R); a prefix match splits them into the
// lower bound in (L, M] (phase 1) and the upper bound in [M, R), kept in
// (HL, HR) until phase 1 ends (phase 2).
// Warps take chunks of worklist entries from one global counter, each
// chunk's base fetched while the previous chunk is handed out.
// Launch bounds: 1024 threads, one CTA per SM, at most 64 registers (no
// spills); smaller CTAs may share an SM up to 1024 threads in all.
template <typename IdxT, bool kSingle>
__global__ void __launch_bounds__(1024, 1) search_kernel(const __grid_constant__ SearchLaunch a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ SmemDesc sdesc[SA_MAX_REFS];
    __shared__ __align__(8) uint64_t mbar;
    const unsigned tid = threadIdx.x;
    const uint32_t n_work = __ldg(a.wl_count);
    if (n_work == 0) return;

    for (unsigned r = tid; r < a.n_refs; r += blockDim.x) {
        const RefDesc &d = a.refs.r[r];
        sdesc[r] = SmemDesc{d.text, d.sa, d.rec, d.krt, d.n, d.smem_off, d.use_depth, d.kmer_k};
    }
    if (tid == 0) {
        mbar_init(&mbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t total = 0;
        for (uint32_t r = 0; r < a.n_refs; r++) {
            const uint32_t d = a.refs.r[r].use_depth;
            if (d) total += table_key_bytes(d) + table_len_bytes(d);
        }
        mbar_arrive_expect_tx(&mbar, total);
        for (uint32_t r = 0; r < a.n_refs; r++) {
            const RefDesc &d = a.refs.r[r];
            if (!d.use_depth) continue;
            bulk_copy_g2s(smem + d.smem_off, d.keys, table_key_bytes(d.use_depth), &mbar);
            bulk_copy_g2s(smem + d.smem_off + table_key_bytes(d.use_depth), d.keylen, table_len_bytes(d.use_depth),
                          &mbar);
        }
    }
    if (!mbar_wait_bounded(&mbar, 0, a.expire_waits ? 0ull : kWaitLimitNs)) {
        if (tid == 0) atomicExch(a.status, SA_ERR_TIMEOUT);
        mbar_wait_bounded(&mbar, 0, kWaitLimitNs);  // let copies in flight land before the CTA exits
        return;
    }

    const unsigned lane = tid & 31u;
    const unsigned lanemask_lt = (1u << lane) - 1u;

    // Reference fields: uniform registers for one reference, else per lane.
    const SmemDesc d0 = sdesc[0];
    const uint64_t *T = d0.text;
    const void *SAp = d0.sa;
    const uint4 *REC = d0.rec;
    const uint4 *KM = d0.krt;
    uint32_t kk = d0.kmer_k;
    uint32_t n = (uint32_t)d0.n;
    const uint8_t *Ktab = smem + d0.off;
    uint32_t depth = d0.depth;

    uint64_t pool_next = 0, pool_end = 0;  // warp-uniform chunk of worklist entries
    unsigned long long pre = 0;             // lane 0: base of the next chunk
    if (lane == 0) pre = atomicAdd(a.counter, (unsigned long long)a.chunk);
    bool exhausted = false;
    bool active = false, fresh = false;
    uint32_t wi = 0, qout = 0, m = 0;
    uint64_t qa = 0, q0 = 0, q1 = 0;
    uint32_t L = 0, R = 0, HL = 0, HR = 0, lcpL = 0, lcpR = 0, hlcpL = 0, hlcpR = 0, lo = 0;
    uint32_t k = 0, phase = 0;

    for (;;) {
        unsigned need = __ballot_sync(0xFFFFFFFFu, !active);
        while (need != 0u && !exhausted) {
            if (pool_next >= pool_end) {
                const unsigned long long base = __shfl_sync(0xFFFFFFFFu, pre, 0);
                if (base >= n_work) {
                    exhausted = true;
                    break;
                }
                pool_next = base;
                pool_end = min((uint64_t)base + a.chunk, (uint64_t)n_work);
                if (lane == 0) pre = atomicAdd(a.counter, (unsigned long long)a.chunk);
            }
            const uint64_t left = pool_end - pool_next;
            const uint32_t avail = left < 32ull ? (uint32_t)left : 32u;
            const uint32_t rank = __popc(need & lanemask_lt);
            if (((need >> lane) & 1u) && rank < avail) {
                wi = (uint32_t)(pool_next + rank);
                active = true;
                fresh = true;
            }
            pool_next += min(avail, (uint32_t)__popc(need));
            need = __ballot_sync(0xFFFFFFFFu, !active);
        }
        if (__ballot_sync(0xFFFFFFFFu, active) == 0u) break;
        if (!active) continue;

        // This iteration's one round of loads: the worklist record (init) or
        // the suffix record at the pivot and query bases 64-127 (deep).
        const bool init = fresh;
        const bool deep = !init && k == 0;
        uint32_t M = L + ((R - L) >> 1);
        const uint4 *wrec = a.wrec + 4 * (size_t)wi;
        uint4 r0, r1;
        ldg32_if(init || deep, init ? (const void *)wrec : (const void *)(REC + 2 * (size_t)M), &r0, &r1);
        // the query's bases 0-63 (init) or 64-127 (deep) from its worklist record
        uint64_t x2 = 0, x3 = 0;
        ldg16_if(init || (deep && m > 64u), wrec + (init ? 2 : 3), &x2, &x3);

        if (init) {
            fresh = false;
            qout = r0.w;
            const uint32_t r = (r1.y >> 16) & 0x7FFFu;
            if (!kSingle) {
                const SmemDesc d = sdesc[r < a.n_refs ? r : 0u];
                T = d.text;
                SAp = d.sa;
                REC = d.rec;
                KM = d.krt;
                kk = d.kmer_k;
                n = (uint32_t)d.n;
                Ktab = smem + d.off;
                depth = d.depth;
            }
            m = r0.z;
            qa = ((uint64_t)(r1.y & 0xFFFFu) << 32) | r1.x;
            q0 = x2;
            q1 = x3;
            lcpL = lcpR = 0;
            phase = 0;
            L = r0.x;
            R = r0.y;
            k = (KM != nullptr && m >= kk) ? 0u : (depth ? 1u : 0u);
            continue;
        }

        int c;
        uint32_t l;
        if (k != 0) {
            // Descent: node k at level lvl samples rank floor((2p+1) n / 2^(lvl+1)).
            const uint32_t lvl = 31u - __clz(k);
            const uint32_t p = k - (1u << lvl);
            M = __umulhi(n, (2u * p + 1u) << (31u - lvl));
            const uint4 kv = reinterpret_cast<const uint4 *>(Ktab)[k];
            const uint32_t klen = Ktab[(16u << depth) + k];
            bool und = false;
            c = cmp_key(q0, q1, m, kv, klen, &l, &und);
            if (und) c = cmp_suffix_tq(T, n, (uint32_t)sa_at<IdxT>(SAp, M), a.tq, qa, m, 64u, &l);
            const uint32_t nk = 2u * k + (c == CMP_GREATER ? 1u : 0u);
            k = (c == CMP_PREFIX || nk >= (1u << depth)) ? 0u : nk;
        } else {
            bool und = false;
            c = cmp_record(q0, q1, x2, x3, m, r0, r1, n, &l, &und);
            if (und) {
                // query bases 96-127 are x3, 128-159 the worklist record's second word pair
                const QueryWindows qw{a.tq, qa, x3, reinterpret_cast<const uint64_t *>(wrec) + 3, 1u};
                c = cmp_suffix_qw(T, n, r1.w, qw, m, max(112u, min(lcpL, lcpR)), &l);
            }
        }
        if (c == CMP_PREFIX && phase == 0) {
            HL = M;
            hlcpL = m;
            HR = R;
            hlcpR = lcpR;
            R = M;
            lcpR = m;
            phase = 1;
            k = 0;
        } else if (c == CMP_LESS || (c == CMP_PREFIX && phase == 1)) {
            R = M;
            lcpR = l;
        } else {
            L = M;
            lcpL = l;
        }
        // Finished intervals: move to the upper bound, or write the result.
        if (R - L <= 1u) {
            if (phase == 1) {
                lo = R;
                L = HL;
                R = HR;
                lcpL = hlcpL;
                lcpR = hlcpR;
                phase = 2;
                k = 0;
            }
            if (R - L <= 1u) {
                const uint32_t lo_out = phase == 0 ? R : lo;
                store_result_sum(a, qout, lo_out, R);
                active = false;
            }
        }
    }
}

// The query (bases qa.. of the packed batch) against the m-prefix of S_p,
// one base at a time (the three cases of Section IV).
__device__ __forceinline__ int cmp_plain(const uint64_t *__restrict__ T, uint64_t n, uint64_t p,
                                         const uint64_t *__restrict__ tq, uint64_t qa, uint32_t m) {
    for (uint32_t k = 0; k < m; k++) {
        if (p + k >= n) return CMP_GREATER;
        const uint64_t b = p + k;
        const uint32_t tb = (uint32_t)(__ldg(T + (b >> 5)) >> (62u - 2u * (uint32_t)(b & 31u))) & 3u;
        const uint64_t c = qa + k;
        const uint32_t qb = (uint32_t)(__ldg(tq + (c >> 5)) >> (62u - 2u * (uint32_t)(c & 31u))) & 3u;
        if (tb != qb) return qb < tb ? CMP_LESS : CMP_GREATER;
    }
    return CMP_PREFIX;
}

template <typename IdxT>
__global__ void __launch_bounds__(256) search_plain_kernel(const __grid_constant__ SearchLaunch a) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.n_q) return;
    uint64_t a0 = __ldg(a.q_off + q) - a.first;
    uint64_t a1 = __ldg(a.q_off + q + 1) - a.first;
    uint32_t r = a.q_ref ? __ldg(a.q_ref + q) : 0u;
    const bool rc = a.revcomp || (a.strand_bits && (r & kStrandBit));
    if (a.strand_bits) r &= ~kStrandBit;
    const bool range_ok = a0 <= a1 && a1 <= a.total && a1 - a0 < (1ull << 31);
    if (range_ok) {  // the other strand sits at the mirrored range of its packing
        const uint64_t len = a1 - a0;
        a0 = strand_start(a0, a1, a.total, rc, a.rc_base);
        a1 = a0 + len;
    }
    bool bad = !range_ok;
    // every base of the query must be one of A, C, G, T (nothing to check in
    // a batch the packing found clean)
    if (range_ok && (a.batch_dirty == nullptr || *a.batch_dirty != 0)) {
        for (uint64_t b = a0; b < a1; b++)
            if ((__ldg(a.tv + (b >> 5)) >> (b & 31u)) & 1u) bad = true;
    }
    if (bad || r >= a.n_refs) {
        if (bad) atomicOr(a.pack_err, 1);
        if (!bad) atomicOr(a.bad_ref, 1);
        store_result_sum(a, q, ~0ull, ~0ull);
        return;
    }
    const uint32_t m = (uint32_t)(a1 - a0);
    const RefDesc &d = a.refs.r[r];
    const uint64_t *T = d.text;
    const uint64_t n = d.n;
    // Lower bound: the first rank whose suffix's m-prefix is not below P.
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (cmp_plain(T, n, sa_at<IdxT>(d.sa, mid), a.tq, a0, m) == CMP_GREATER)
            lo = mid + 1;
        else
            hi = mid;
    }
    const uint64_t first = lo;
    // Upper bound: the first rank whose suffix's m-prefix is above P.
    hi = n;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (cmp_plain(T, n, sa_at<IdxT>(d.sa, mid), a.tq, a0, m) != CMP_LESS)
            lo = mid + 1;
        else
            hi = mid;
    }
    store_result_sum(a, q, first, lo);
}

__global__ void search_status_kernel(const int *flags, int *dst) {
    int st = flags[1];
    if (st == 0 && flags[0]) st = SA_ERR_BASE;
    if (st == 0 && flags[3]) st = SA_ERR_ARG;
    *dst = st;
}

__global__ void capacity_status_kernel(const int *overflow, int *dst) {
    if (*overflow && *dst == SA_OK) *dst = SA_ERR_CAPACITY;
}

// Precedence of statuses across the chunks of one call: a wait that ran out,
// then a byte that is not a base, then a bad reference id.
__device__ __forceinline__ int status_rank(int st) {
    return st == SA_ERR_TIMEOUT ? 3 : st == SA_ERR_BASE ? 2 : st == SA_ERR_ARG ? 1 : 0;
}

__global__ void fold_status_kernel(const int *flags, int *acc) {
    int st = flags[1];
    if (st == 0 && flags[0]) st = SA_ERR_BASE;
    if (st == 0 && flags[3]) st = SA_ERR_ARG;
    atomicMax(acc, status_rank(st));
}

__global__ void fold_final_kernel(const int *acc, bool check_overflow, int *dst) {
    const int rank = acc[0];
    int st = rank == 3 ? SA_ERR_TIMEOUT : rank == 2 ? SA_ERR_BASE : rank == 1 ? SA_ERR_ARG : SA_OK;
    if (st == SA_OK && check_overflow && acc[1]) st = SA_ERR_CAPACITY;
    *dst = st;
}

}  // namespace

cudaError_t launch_search_status(const int *flags, int *dst, cudaStream_t s) {
    search_status_kernel<<<1, 1, 0, s>>>(flags, dst);
    return cudaGetLastError();
}

cudaError_t launch_fold_status(const int *flags, int *acc, cudaStream_t s) {
    fold_status_kernel<<<1, 1, 0, s>>>(flags, acc);
    return cudaGetLastError();
}

cudaError_t launch_fold_final(const int *acc, bool check_overflow, int *dst, cudaStream_t s) {
    fold_final_kernel<<<1, 1, 0, s>>>(acc, check_overflow, dst);
    return cudaGetLastError();
}

cudaError_t launch_capacity_status(const int *overflow, int *dst, cudaStream_t s) {
    capacity_status_kernel<<<1, 1, 0, s>>>(overflow, dst);
    return cudaGetLastError();
}

cudaError_t launch_search(const SearchLaunch &L, cudaStream_t s) {
    if (L.n_q == 0) return cudaSuccess;
    const size_t smem = L.smem_bytes;
    const bool single = L.n_refs == 1 && L.q_ref == nullptr;
    auto go = [&](auto kernel) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kernel<<<L.blocks, L.threads, smem, s>>>(L);
    };
    auto pick = [&](auto idx_tag, auto single_tag) {
        using I = decltype(idx_tag);
        constexpr bool S = decltype(single_tag)::value;
        go(search_kernel<I, S>);
    };
    if (L.width == 4)
        single ? pick(uint32_t{}, std::true_type{}) : pick(uint32_t{}, std::false_type{});
    else
        single ? pick(uint64_t{}, std::true_type{}) : pick(uint64_t{}, std::false_type{});
    return cudaGetLastError();
}

cudaError_t launch_search_plain(const SearchLaunch &L, cudaStream_t s) {
    if (L.n_q == 0) return cudaSuccess;
    const uint64_t blocks = (L.n_q + 255) / 256;
    if (L.width == 4)
        search_plain_kernel<uint32_t><<<(unsigned)blocks, 256, 0, s>>>(L);
    else
        search_plain_kernel<uint64_t><<<(unsigned)blocks, 256, 0, s>>>(L);
    return cudaGetLastError();
}

uint32_t search_table_bytes(uint32_t depth) { return depth ? table_key_bytes(depth) + table_len_bytes(depth) : 0u; }

}  // namespace sa
