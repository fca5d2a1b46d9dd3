// build.cu -- suffix-array construction on the GPU by prefix doubling (or the
// upload of one built on the host by DC3), and the sampled-key table.  Off the
// search path; timed apart from it.
//
// The paper builds its suffix array on the host (the straightforward sort or
// DC3, Section III).  Here the text is already packed in device memory, so
// the array is built there: every suffix is first ranked by its first 29
// bases (58 bits of packed text plus a 6-bit length that puts a proper prefix
// first, the order of Table I).  Then, while some group of equal ranks has
// more than one member, only the members of such groups are re-sorted by the
// pair (rank[i], rank[i + h]) and h doubles.  Ranks are the suffix-array
// position of the first member of the group, so they order groups globally
// and a finished group's rank is its final position.  The radix sorts, scans
// and compactions come from CUB (a source-only library shipped with the CUDA
// toolkit); the key computation, rank scatter and key table are kernels here.
#include <cub/cub.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <vector>

#include "dc3.h"
#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kThreads = 256;

unsigned grid_for(uint64_t n) {
    uint64_t b = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)device_sm_count() * 32;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

#define GS_LOOP(i, n) \
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

// Initial key of suffix i: its first 29 bases, then min(29, n - i).  Bits past
// the text are zero, so equal packed prefixes are ordered by length.
__global__ void init_keys_kernel(const uint64_t *__restrict__ T, uint64_t n, uint64_t *keys, uint32_t *vals) {
    GS_LOOP(i, n) {
        const uint64_t w = text_window(T, i);
        const uint64_t len = (n - i) < 29 ? (n - i) : 29;
        keys[i] = (w & ~0x3Full) | len;
        vals[i] = (uint32_t)i;
    }
}

// head value: j if position j starts a group of equal keys, else 0.
__global__ void head_values_kernel(const uint64_t *__restrict__ keys, uint64_t cnt,
                                   const uint32_t *__restrict__ pos, uint32_t *hv) {
    GS_LOOP(t, cnt) {
        const bool head = t == 0 || keys[t] != keys[t - 1];
        hv[t] = head ? (pos ? pos[t] : (uint32_t)t) : 0u;
    }
}

// After the scan, rank[t] is the SA position of t's group head.  Writes the
// ranks, the suffix-array entries, and flags members of groups of size > 1.
__global__ void scatter_ranks_kernel(const uint64_t *__restrict__ keys, uint64_t cnt,
                                     const uint32_t *__restrict__ pos,   // SA positions (null = identity)
                                     const uint32_t *__restrict__ sorted_vals, const uint32_t *__restrict__ rank,
                                     uint32_t *isa, uint32_t *sa, uint8_t *unresolved) {
    GS_LOOP(t, cnt) {
        const uint32_t i = sorted_vals[t];
        const uint32_t j = pos ? pos[t] : (uint32_t)t;
        sa[j] = i;
        isa[i] = rank[t];
        const bool head = t == 0 || keys[t] != keys[t - 1];
        const bool tail = t + 1 == cnt || keys[t + 1] != keys[t];
        unresolved[t] = (head && tail) ? 0 : 1;
    }
}

// Doubling key of the unresolved member at SA position pos[t].
__global__ void pair_keys_kernel(const uint32_t *__restrict__ pos, uint64_t cnt, const uint32_t *__restrict__ sa,
                                 const uint32_t *__restrict__ isa, uint64_t n, uint64_t h, uint64_t *keys,
                                 uint32_t *vals) {
    GS_LOOP(t, cnt) {
        const uint32_t i = sa[pos[t]];
        const uint64_t r1 = isa[i];
        const uint64_t r2 = (uint64_t)i + h < n ? (uint64_t)isa[i + h] + 1 : 0;
        keys[t] = (r1 << 32) | r2;
        vals[t] = i;
    }
}

__global__ void widen_kernel(const uint32_t *__restrict__ src, uint64_t n, uint64_t *dst) {
    GS_LOOP(i, n) dst[i] = src[i];
}

struct MaxOp {
    __device__ __forceinline__ uint32_t operator()(uint32_t a, uint32_t b) const { return a > b ? a : b; }
};

int bit_length(uint64_t x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

struct Pool {
    cudaStream_t s;
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (err != cudaSuccess) return nullptr;
        err = scratch_alloc(&p, count * sizeof(T) + 16, s);
        if (err == cudaSuccess) ptrs.push_back(p);
        return reinterpret_cast<T *>(p);
    }
    ~Pool() {
        for (void *p : ptrs) scratch_free(p, s);
    }
};

}  // namespace

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return status_from_cuda(e_); \
    } while (0)

int build_suffix_array(sa_index *idx, cudaStream_t s) {
    const uint64_t n = idx->n;
    Pool pool{s};
    uint64_t *kA = pool.get<uint64_t>(n), *kB = pool.get<uint64_t>(n);
    uint32_t *vA = pool.get<uint32_t>(n), *vB = pool.get<uint32_t>(n);
    uint32_t *isa = pool.get<uint32_t>(n), *sa32 = pool.get<uint32_t>(n);
    uint32_t *hv = pool.get<uint32_t>(n), *rank = pool.get<uint32_t>(n);
    uint32_t *posA = pool.get<uint32_t>(n), *posB = pool.get<uint32_t>(n);
    uint8_t *flag = pool.get<uint8_t>(n);
    uint64_t *d_count = pool.get<uint64_t>(1);
    if (pool.err != cudaSuccess) return SA_ERR_NOMEM;

    // Temporary storage sized for the largest call of each CUB routine.
    size_t t_sort = 0, t_scan = 0, t_sel = 0, t_sel0 = 0;
    thrust::counting_iterator<uint32_t> iota(0);
    {
        cub::DoubleBuffer<uint64_t> kb(kA, kB);
        cub::DoubleBuffer<uint32_t> vb(vA, vB);
        CK(cub::DeviceRadixSort::SortPairs(nullptr, t_sort, kb, vb, n, 0, 64, s));
        CK(cub::DeviceScan::InclusiveScan(nullptr, t_scan, hv, rank, MaxOp(), n, s));
        CK(cub::DeviceSelect::Flagged(nullptr, t_sel, posA, flag, posB, d_count, n, s));
        CK(cub::DeviceSelect::Flagged(nullptr, t_sel0, iota, flag, posB, d_count, n, s));
    }
    size_t t_bytes = t_sort > t_scan ? t_sort : t_scan;
    if (t_sel > t_bytes) t_bytes = t_sel;
    if (t_sel0 > t_bytes) t_bytes = t_sel0;
    void *temp = pool.get<uint8_t>(t_bytes);
    if (pool.err != cudaSuccess) return SA_ERR_NOMEM;

    const unsigned g = grid_for(n);
    // Round 0: rank by the first 29 bases.
    init_keys_kernel<<<g, kThreads, 0, s>>>(idx->text, n, kA, vA);
    CK(cudaGetLastError());
    cub::DoubleBuffer<uint64_t> kb(kA, kB);
    cub::DoubleBuffer<uint32_t> vb(vA, vB);
    CK(cub::DeviceRadixSort::SortPairs(temp, t_bytes, kb, vb, n, 0, 64, s));
    head_values_kernel<<<g, kThreads, 0, s>>>(kb.Current(), n, nullptr, hv);
    CK(cudaGetLastError());
    CK(cub::DeviceScan::InclusiveScan(temp, t_bytes, hv, rank, MaxOp(), n, s));
    scatter_ranks_kernel<<<g, kThreads, 0, s>>>(kb.Current(), n, nullptr, vb.Current(), rank, isa, sa32, flag);
    CK(cudaGetLastError());
    // Unresolved SA positions, in increasing order.
    CK(cub::DeviceSelect::Flagged(temp, t_bytes, iota, flag, posA, d_count, n, s));
    uint64_t cnt = 0;
    CK(cudaMemcpyAsync(&cnt, d_count, sizeof cnt, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));

    const int rank_bits = bit_length(n);
    uint64_t h = 29;
    uint32_t *pos = posA, *pos_next = posB;
    while (cnt > 0) {
        const unsigned gc = grid_for(cnt);
        pair_keys_kernel<<<gc, kThreads, 0, s>>>(pos, cnt, sa32, isa, n, h, kA, vA);
        CK(cudaGetLastError());
        cub::DoubleBuffer<uint64_t> rk(kA, kB);
        cub::DoubleBuffer<uint32_t> rv(vA, vB);
        CK(cub::DeviceRadixSort::SortPairs(temp, t_bytes, rk, rv, cnt, 0, 32 + rank_bits, s));
        head_values_kernel<<<gc, kThreads, 0, s>>>(rk.Current(), cnt, pos, hv);
        CK(cudaGetLastError());
        CK(cub::DeviceScan::InclusiveScan(temp, t_bytes, hv, rank, MaxOp(), cnt, s));
        scatter_ranks_kernel<<<gc, kThreads, 0, s>>>(rk.Current(), cnt, pos, rv.Current(), rank, isa, sa32, flag);
        CK(cudaGetLastError());
        CK(cub::DeviceSelect::Flagged(temp, t_bytes, pos, flag, pos_next, d_count, cnt, s));
        CK(cudaMemcpyAsync(&cnt, d_count, sizeof cnt, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        uint32_t *tmp = pos;
        pos = pos_next;
        pos_next = tmp;
        h *= 2;
    }
    if (idx->width == 4) {
        CK(cudaMemcpyAsync(idx->sa, sa32, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    } else {
        widen_kernel<<<g, kThreads, 0, s>>>(sa32, n, reinterpret_cast<uint64_t *>(idx->sa));
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(s));
    return SA_OK;
}

// The suffix array built on the host by DC3 (Section III's construction, in
// dc3_host.cpp) from host_text, then uploaded (and widened for 64-bit
// indexes on the device).
int build_suffix_array_host(sa_index *idx, const char *host_text, void *stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t n = idx->n;
    std::vector<uint32_t> sa32;
    try {
        sa32.resize(n);
    } catch (const std::bad_alloc &) {
        return SA_ERR_NOMEM;
    }
    const int st = dc3_suffix_array(host_text, n, sa32.data());
    if (st != SA_OK) return st;
    if (idx->width == 4) {
        CK(cudaMemcpyAsync(idx->sa, sa32.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    } else {
        Pool pool{s};
        uint32_t *d = pool.get<uint32_t>(n);
        if (pool.err != cudaSuccess) return SA_ERR_NOMEM;
        CK(cudaMemcpyAsync(d, sa32.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        widen_kernel<<<grid_for(n), kThreads, 0, s>>>(d, n, reinterpret_cast<uint64_t *>(idx->sa));
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    }
    return SA_OK;
}

// Key table in level (breadth-first) order: node k >= 1 at level l = floor(log2 k),
// p = k - 2^l, samples rank floor((2p + 1) n / 2^(l+1)).  Its first 2^d - 1
// nodes are the table of depth d, so a shallower table is a prefix.  Entry k
// holds the first 64 bases of that suffix (bits past the text are zero) and
// keylen[k] = min(64, n - SA[rank]).  Node 0 is unused padding.
template <typename IdxT>
__global__ void build_keys_kernel(const uint64_t *__restrict__ T, const IdxT *__restrict__ sa, uint64_t n,
                                  uint32_t depth, uint32_t entries, uint4 *keys, uint8_t *keylen) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < entries; k += gridDim.x * blockDim.x) {
        uint64_t w0 = 0, w1 = 0;
        uint32_t len = 0;
        if (k >= 1 && k < (1u << depth)) {
            const uint32_t l = 31 - __clz(k);
            const uint64_t p = k - (1u << l);
            const uint64_t rank = ((2 * p + 1) * n) >> (l + 1);
            const uint64_t pos = sa[rank];
            w0 = text_window(T, pos);
            w1 = text_window(T, pos + 32);
            const uint64_t rem = n - pos;
            len = rem < 64 ? (uint32_t)rem : 64u;
        }
        keys[k] = make_uint4((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1, (uint32_t)(w1 >> 32));
        keylen[k] = (uint8_t)len;
    }
}

cudaError_t launch_build_keys(sa_index *idx, cudaStream_t s) {
    const uint32_t entries = idx->depth >= 4 ? (1u << idx->depth) : 16u;
    const unsigned blocks = (entries + 255) / 256;
    if (idx->width == 4)
        build_keys_kernel<uint32_t><<<blocks, 256, 0, s>>>(idx->text, reinterpret_cast<const uint32_t *>(idx->sa),
                                                           idx->n, idx->depth, entries, idx->keys, idx->keylen);
    else
        build_keys_kernel<uint64_t><<<blocks, 256, 0, s>>>(idx->text, reinterpret_cast<const uint64_t *>(idx->sa),
                                                           idx->n, idx->depth, entries, idx->keys, idx->keylen);
    return cudaGetLastError();
}

// Suffix records: for rank i, the first 112 bases of suffix SA[i] and SA[i]
// itself in one 32-byte entry (one DRAM sector), so that a probe of the
// search reads one aligned sector instead of an SA entry and then the text it
// points to, and a query of up to 112 bases never reads the text.
template <typename IdxT>
__global__ void build_records_kernel(const uint64_t *__restrict__ T, const IdxT *__restrict__ sa, uint64_t n,
                                     uint4 *rec) {
    GS_LOOP(i, n) {
        const uint64_t pos = sa[i];
        const uint64_t w0 = text_window(T, pos);
        const uint64_t w1 = text_window(T, pos + 32);
        const uint64_t w2 = text_window(T, pos + 64);
        const uint64_t w3 = text_window(T, pos + 96);
        rec[2 * i] = make_uint4((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1, (uint32_t)(w1 >> 32));
        rec[2 * i + 1] = make_uint4((uint32_t)w2, (uint32_t)(w2 >> 32), (uint32_t)(w3 >> 32), (uint32_t)pos);
    }
}

// k-mer table.  For rank i let f(i) be the smallest k-base string x with
// S_SA[i] < x: the suffix's k-base prefix plus one when it has k bases or
// more, else the suffix padded with A (a suffix that is a proper prefix of x
// sorts before x).  f is non-decreasing along the suffix array, and
// kmer[x] = #{i : f(i) <= x} = #{suffixes sorting before x}.  Thread i writes
// kmer[x] = i for f(i-1) <= x < f(i), with f(-1) = 0 and f(n) = 4^k + 1, so
// every entry is written once.
__device__ __forceinline__ uint64_t kmer_f(const uint4 *rec, uint64_t i, uint64_t n, uint32_t k) {
    const uint4 r0 = rec[2 * i];
    const uint32_t pos = rec[2 * i + 1].w;
    const uint64_t w0 = ((uint64_t)r0.y << 32) | r0.x;
    const uint64_t x = w0 >> (64u - 2u * k);
    return (n - pos) >= k ? x + 1 : x;
}

__global__ void build_kmer_kernel(const uint4 *__restrict__ rec, uint64_t n, uint32_t k, uint32_t *kmer) {
    const uint64_t top = (1ull << (2 * k)) + 1;
    GS_LOOP(i, n + 1) {
        const uint64_t fa = i == 0 ? 0 : kmer_f(rec, i - 1, n, k);
        const uint64_t fb = i == n ? top : kmer_f(rec, i, n, k);
        for (uint64_t x = fa; x < fb; x++) kmer[x] = (uint32_t)i;
    }
}

// k-mer table entry, 64 bytes (4 uint4) per k-base string x:
//   {lo, hi, pos, clamp}: ranks [lo, hi) hold the suffixes that sort at or
//     after x and before x + 1 (those with prefix x, and any suffix shorter
//     than k that falls between the two), lo = number of suffixes sorting
//     before x; when hi > lo, pos is the position of the suffix at rank
//     M = lo - 1 + (hi - lo + 1) / 2 -- the first pivot of the lockstep binary
//     search over (lo - 1, hi) -- and clamp = min(192, n - pos) the number of
//     its first 192 bases that exist;
//   three uint4: the first 192 bases of that suffix as six packed words.
// One aligned 64-byte read therefore brackets a query of m >= k bases and
// makes its first probe.
__global__ void build_krt_kernel(const uint32_t *__restrict__ kmer, const uint4 *__restrict__ rec,
                                 const uint64_t *__restrict__ T, uint64_t n, uint32_t k, uint4 *__restrict__ krt) {
    const uint64_t entries = 1ull << (2 * k);
    GS_LOOP(x, entries) {
        const uint32_t lo = kmer[x], hi = kmer[x + 1];
        uint4 h = make_uint4(lo, hi, 0u, 0u);
        uint64_t e[6] = {0, 0, 0, 0, 0, 0};
        if (hi > lo) {
            const uint32_t M = lo + (hi - lo + 1u) / 2u - 1u;
            const uint64_t pos = rec[2 * (uint64_t)M + 1].w;
            const uint64_t left = n - pos;  // >= 1
            h.z = (uint32_t)pos;
            h.w = (uint32_t)(left < 192 ? left : 192);
#pragma unroll
            for (int j = 0; j < 6; j++) {
                const uint64_t b = pos + 32ull * j;
                e[j] = b < n ? text_window(T, b) : 0ull;
            }
        }
        uint4 *dst = krt + 4 * x;
        dst[0] = h;
        dst[1] = make_uint4((uint32_t)e[0], (uint32_t)(e[0] >> 32), (uint32_t)e[1], (uint32_t)(e[1] >> 32));
        dst[2] = make_uint4((uint32_t)e[2], (uint32_t)(e[2] >> 32), (uint32_t)e[3], (uint32_t)(e[3] >> 32));
        dst[3] = make_uint4((uint32_t)e[4], (uint32_t)(e[4] >> 32), (uint32_t)e[5], (uint32_t)(e[5] >> 32));
    }
}

// The plain counts kmer[x] = lo of every entry, and kmer[4^k] = n.
__global__ void krt_lo_kernel(const uint4 *__restrict__ krt, uint64_t n, uint32_t k, uint32_t *__restrict__ out) {
    const uint64_t entries = 1ull << (2 * k);
    GS_LOOP(x, entries + 1) out[x] = x < entries ? krt[4 * x].x : (uint32_t)n;
}

cudaError_t launch_build_kmer(sa_index *idx, cudaStream_t s) {
    if (!idx->krt) return cudaSuccess;
    const uint64_t entries = 1ull << (2 * idx->kmer_k);
    uint32_t *kmer = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void **>(&kmer), (entries + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    build_kmer_kernel<<<grid_for(idx->n + 1), kThreads, 0, s>>>(idx->rec, idx->n, idx->kmer_k, kmer);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        build_krt_kernel<<<grid_for(entries), kThreads, 0, s>>>(kmer, idx->rec, idx->text, idx->n, idx->kmer_k,
                                                                idx->krt);
        e = cudaGetLastError();
    }
    scratch_free(kmer, s);
    return e;
}

cudaError_t launch_copy_kmer_counts(const sa_index *idx, uint32_t *dst, cudaStream_t s) {
    const uint64_t entries = 1ull << (2 * idx->kmer_k);
    krt_lo_kernel<<<grid_for(entries + 1), kThreads, 0, s>>>(idx->krt, idx->n, idx->kmer_k, dst);
    return cudaGetLastError();
}

cudaError_t launch_build_records(sa_index *idx, cudaStream_t s) {
    const unsigned g = grid_for(idx->n);
    if (idx->width == 4)
        build_records_kernel<uint32_t><<<g, kThreads, 0, s>>>(idx->text, reinterpret_cast<const uint32_t *>(idx->sa),
                                                              idx->n, idx->rec);
    else
        build_records_kernel<uint64_t><<<g, kThreads, 0, s>>>(idx->text, reinterpret_cast<const uint64_t *>(idx->sa),
                                                              idx->n, idx->rec);
    return cudaGetLastError();
}

}  // namespace sa
