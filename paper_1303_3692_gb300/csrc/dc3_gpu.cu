// dc3_gpu.cu -- the suffix array on the GPU by the construction Section III
// describes: the difference cover modulo 3 (DC3, the skew algorithm of
// Kärkkäinen and Sanders).  The steps are those of dc3_host.cpp, each a
// data-parallel pass:
//   1. the sample suffixes start at i mod 3 != 0 (plus the empty suffix at
//      i = n when n mod 3 == 1, so that the mod-1 part of the reduced string
//      ends in a unique letter);
//   2. the samples are sorted by their first three letters (radix sorts; one
//      pass on a packed key when three letters fit 64 bits) and each distinct
//      triple is named by its rank (Table II ranks the samples this way); when
//      two samples share a name, the suffix array of the reduced string --
//      the names of the mod-1 samples in text order, then of the mod-2 ones --
//      orders them, computed by the same construction one level down;
//   3. the mod-0 suffixes are sorted by (letter, rank of the sample at i + 1)
//      (Section III's B0 example: S9 <= S0 <= S6 <= S3): the mod-1 samples in
//      rank order give them sorted by the second key, and a stable radix sort
//      by the letter finishes;
//   4. the two sorted lists are merged: a mod-0 suffix and a sample compare
//      by at most two letters and one sample rank, so each suffix's key (two
//      letters, two ranks) is gathered once into a 16-byte record in list
//      order, and the merge streams the records (merge path: each thread
//      finds where its run of 32 outputs starts by a binary search on its
//      diagonal, then merges the run).
// The radix sorts, scans and compactions come from CUB; the rest are kernels
// here.  The top level reads its letters (codes 1..4, 0 past the end) from the
// packed text, so the text is never unpacked.
#include <cub/cub.cuh>
#include <vector>

#include "sa_internal.cuh"

namespace sa {

namespace {

constexpr int kThreads = 256;

unsigned grid_of(uint64_t n) {
    uint64_t b = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)device_sm_count() * 32;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

#define DC3_LOOP(i, n) \
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (uint64_t)gridDim.x * blockDim.x)

// The top level's letters: base codes 1..4 from the packed text, 0 past the end.
struct PackedLetters {
    const uint64_t *T;
    uint64_t n;
    __device__ __forceinline__ uint32_t operator()(uint64_t i) const {
        return i < n ? (uint32_t)((__ldg(T + (i >> 5)) >> (62u - 2u * (uint32_t)(i & 31u))) & 3u) + 1u : 0u;
    }
};

// A deeper level's letters: the names of the level above, 0 past the end.
struct NameLetters {
    const uint32_t *s;
    uint64_t n;
    __device__ __forceinline__ uint32_t operator()(uint64_t i) const { return i < n ? __ldg(s + i) : 0u; }
};

// Index of sample position p in the reduced string (mod-1 samples first).
__device__ __forceinline__ uint64_t ridx(uint64_t p, uint64_t n0) { return p % 3 == 1 ? (p - 1) / 3 : n0 + (p - 2) / 3; }

__device__ __forceinline__ uint64_t sample_pos(uint64_t j, uint64_t n0) { return j < n0 ? 3 * j + 1 : 3 * (j - n0) + 2; }

__global__ void init_samples_kernel(uint32_t *pos, uint64_t n0, uint64_t n02) {
    DC3_LOOP(j, n02) pos[j] = (uint32_t)sample_pos(j, n0);
}

// Packed key of three letters of `bits` bits each (3 * bits <= 64).
template <typename L>
__global__ void triple_key_kernel(L s, const uint32_t *__restrict__ pos, uint64_t m, uint32_t bits, uint64_t *key) {
    DC3_LOOP(t, m) {
        const uint64_t p = pos[t];
        key[t] = ((uint64_t)s(p) << (2 * bits)) | ((uint64_t)s(p + 1) << bits) | (uint64_t)s(p + 2);
    }
}

// One letter of every position: key[t] = s(pos[t] + off).
template <typename L>
__global__ void letter_key_kernel(L s, const uint32_t *__restrict__ pos, uint64_t m, uint32_t off, uint32_t *key) {
    DC3_LOOP(t, m) key[t] = s((uint64_t)pos[t] + off);
}

// flag[t] = 1 where the triple at sorted position t differs from the one before.
template <typename L>
__global__ void new_name_kernel(L s, const uint32_t *__restrict__ pos, uint64_t m, uint32_t *flag) {
    DC3_LOOP(t, m) {
        uint32_t f = 1;
        if (t > 0) {
            const uint64_t p = pos[t], q = pos[t - 1];
            f = (s(p) != s(q) || s(p + 1) != s(q + 1) || s(p + 2) != s(q + 2)) ? 1u : 0u;
        }
        flag[t] = f;
    }
}

// red[ridx(pos[t])] = name[t]: the reduced string.
__global__ void scatter_names_kernel(const uint32_t *__restrict__ pos, const uint32_t *__restrict__ name, uint64_t m,
                                     uint64_t n0, uint32_t *red) {
    DC3_LOOP(t, m) red[ridx(pos[t], n0)] = name[t];
}

// red[sar[r]] = r + 1: each sample's rank from the suffix array of the reduced string.
__global__ void ranks_of_kernel(const uint32_t *__restrict__ sar, uint64_t m, uint32_t *red) {
    DC3_LOOP(r, m) red[sar[r]] = (uint32_t)(r + 1);
}

// s12[r] = position of the sample at rank r + 1, read off the reduced
// string's suffix array (whose r-th entry is that sample's index).
__global__ void samples_in_order_kernel(const uint32_t *__restrict__ sar, uint64_t n0, uint64_t n02, uint32_t *s12) {
    DC3_LOOP(r, n02) s12[r] = (uint32_t)sample_pos(__ldg(sar + r), n0);
}

// The predecessors of the mod-1 samples, in the samples' rank order.
__global__ void mod0_candidates_kernel(const uint32_t *__restrict__ s12, uint64_t m, uint32_t *cand, uint8_t *flag) {
    DC3_LOOP(r, m) {
        const uint32_t p = s12[r];
        flag[r] = p % 3 == 1 ? 1 : 0;
        cand[r] = p - 1;
    }
}

// The merge of the mod-0 list A and the sample list B (without the empty
// sample).  A mod-0 suffix a and a sample b compare by at most two letters and
// one sample rank: a's key is {s(a), s(a+1), rank(a+1), rank(a+2)}; a mod-1
// sample's {s(b), -, rank(b+1), -}; a mod-2 sample's {s(b), s(b+1), -,
// rank(b+2)} (the rank of the suffix past the end is 0, below every sample).
// The keys are gathered once (merge_keys_kernel: the random reads of the
// merge), so that the merge itself streams them.
template <typename L>
struct KeyOf {
    L s;
    const uint32_t *red;  // 1-based sample ranks
    uint64_t n, n0;
    __device__ __forceinline__ uint32_t rank(uint64_t p) const { return p >= n ? 0u : __ldg(red + ridx(p, n0)); }
    __device__ __forceinline__ uint4 operator()(uint64_t p) const {
        const uint32_t m = (uint32_t)(p % 3);
        return make_uint4(s(p), m == 1 ? 0u : s(p + 1), m == 2 ? 0u : rank(p + 1), m == 1 ? 0u : rank(p + 2));
    }
};

template <typename L>
__global__ void merge_keys_kernel(KeyOf<L> key, const uint32_t *__restrict__ P, uint64_t np, uint4 *K) {
    DC3_LOOP(i, np) K[i] = key(__ldg(P + i));
}

// Is the mod-0 suffix with key ka before the sample with key kb (kb_mod1: the
// sample is a mod-1 one)?
__device__ __forceinline__ bool key_before(uint4 ka, uint4 kb, bool kb_mod1) {
    if (ka.x != kb.x) return ka.x < kb.x;
    if (kb_mod1) return ka.z < kb.z;
    if (ka.y != kb.y) return ka.y < kb.y;
    return ka.w < kb.w;
}

constexpr int kMergeItems = 32;

__global__ void merge_kernel(const uint4 *__restrict__ KA, const uint32_t *__restrict__ A, uint64_t na,
                             const uint4 *__restrict__ KB, const uint32_t *__restrict__ B, uint64_t nb,
                             uint32_t *out) {
    const uint64_t total = na + nb;
    DC3_LOOP(tid, (total + kMergeItems - 1) / kMergeItems) {
        const uint64_t d = tid * kMergeItems;
        // co-rank: how many of the first d outputs come from A
        uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
        while (lo < hi) {
            const uint64_t i = (lo + hi) / 2, j = d - i - 1;
            if (key_before(__ldg(KA + i), __ldg(KB + j), __ldg(B + j) % 3 == 1))
                lo = i + 1;
            else
                hi = i;
        }
        uint64_t i = lo, j = d - lo;
        const uint64_t end = d + kMergeItems < total ? d + kMergeItems : total;
        uint4 ka = i < na ? __ldg(KA + i) : make_uint4(0, 0, 0, 0);
        uint4 kb = j < nb ? __ldg(KB + j) : make_uint4(0, 0, 0, 0);
        uint32_t pb = j < nb ? __ldg(B + j) : 0u;
        for (uint64_t o = d; o < end; o++) {
            if (j >= nb || (i < na && key_before(ka, kb, pb % 3 == 1))) {
                out[o] = __ldg(A + i);
                if (++i < na) ka = __ldg(KA + i);
            } else {
                out[o] = pb;
                if (++j < nb) {
                    kb = __ldg(KB + j);
                    pb = __ldg(B + j);
                }
            }
        }
    }
}

__global__ void widen_sa_kernel(const uint32_t *__restrict__ src, uint64_t n, uint64_t *dst) { DC3_LOOP(i, n) dst[i] = src[i]; }

int bits_of(uint64_t x) {
    int b = 0;
    while (x) {
        b++;
        x >>= 1;
    }
    return b;
}

// Device scratch of one level; buffers can be released early (stream-ordered).
struct LevelScratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    bool failed = false;
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (failed) return nullptr;
        if (scratch_alloc(&p, count * sizeof(T) + 16, s) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return nullptr;
        }
        ptrs.push_back(p);
        return reinterpret_cast<T *>(p);
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) {
                scratch_free(q, s);
                q = nullptr;
            }
    }
    ~LevelScratch() {
        for (void *p : ptrs)
            if (p) scratch_free(p, s);
    }
};

#define DC3_CK(x)                                            \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) return status_from_cuda(e_);  \
    } while (0)

// Stable sort of the positions pos[0..m) by key (a double buffer each);
// returns the sorted positions' buffer.
template <typename K>
int radix_by_key(cub::DoubleBuffer<K> &key, cub::DoubleBuffer<uint32_t> &pos, uint64_t m, int end_bit, cudaStream_t s,
                 LevelScratch &sc) {
    size_t tb = 0;
    DC3_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, key, pos, m, 0, end_bit, s));
    void *temp = sc.get<uint8_t>(tb);
    if (!temp) return SA_ERR_NOMEM;
    DC3_CK(cub::DeviceRadixSort::SortPairs(temp, tb, key, pos, m, 0, end_bit, s));
    sc.release(temp);
    return SA_OK;
}

// The suffix array of the string s[0..n) over letters [1, K] (0 past the
// end) into sa[0..n).
template <typename L>
int skew_gpu(L s, uint64_t n, uint32_t K, uint32_t *sa, cudaStream_t st) {
    const uint64_t n0 = (n + 2) / 3, n2 = n / 3, n02 = n0 + n2;
    const int lb = bits_of(K);  // bits of a letter (letters 0..K)
    LevelScratch sc{st};

    // Step 2: the samples sorted by their leading triple, and named.
    uint32_t *red = sc.get<uint32_t>(n02);
    uint32_t *sorted = nullptr;  // sample positions in triple order
    uint32_t *posA = sc.get<uint32_t>(n02), *posB = sc.get<uint32_t>(n02);
    if (sc.failed) return SA_ERR_NOMEM;
    init_samples_kernel<<<grid_of(n02), kThreads, 0, st>>>(posA, n0, n02);
    DC3_CK(cudaGetLastError());
    cub::DoubleBuffer<uint32_t> pb(posA, posB);
    if (3 * lb <= 64) {
        uint64_t *kA = sc.get<uint64_t>(n02), *kB = sc.get<uint64_t>(n02);
        if (sc.failed) return SA_ERR_NOMEM;
        triple_key_kernel<<<grid_of(n02), kThreads, 0, st>>>(s, posA, n02, (uint32_t)lb, kA);
        DC3_CK(cudaGetLastError());
        cub::DoubleBuffer<uint64_t> kb(kA, kB);
        int r = radix_by_key(kb, pb, n02, 3 * lb, st, sc);
        if (r) return r;
        sc.release(kA);
        sc.release(kB);
    } else {  // least significant letter first; the sorts are stable
        uint32_t *kA = sc.get<uint32_t>(n02), *kB = sc.get<uint32_t>(n02);
        if (sc.failed) return SA_ERR_NOMEM;
        for (int off = 2; off >= 0; off--) {
            letter_key_kernel<<<grid_of(n02), kThreads, 0, st>>>(s, pb.Current(), n02, (uint32_t)off, kA);
            DC3_CK(cudaGetLastError());
            cub::DoubleBuffer<uint32_t> kb(kA, kB);
            int r = radix_by_key(kb, pb, n02, lb, st, sc);
            if (r) return r;
        }
        sc.release(kA);
        sc.release(kB);
    }
    sorted = pb.Current();
    uint32_t *other = pb.Alternate();
    // names: an inclusive scan of "differs from the triple before"
    new_name_kernel<<<grid_of(n02), kThreads, 0, st>>>(s, sorted, n02, other);
    DC3_CK(cudaGetLastError());
    {
        size_t tb = 0;
        DC3_CK(cub::DeviceScan::InclusiveSum(nullptr, tb, other, other, n02, st));
        void *temp = sc.get<uint8_t>(tb);
        if (!temp) return SA_ERR_NOMEM;
        DC3_CK(cub::DeviceScan::InclusiveSum(temp, tb, other, other, n02, st));
        sc.release(temp);
    }
    scatter_names_kernel<<<grid_of(n02), kThreads, 0, st>>>(sorted, other, n02, n0, red);
    DC3_CK(cudaGetLastError());
    uint32_t names = 0;
    DC3_CK(cudaMemcpyAsync(&names, other + (n02 - 1), sizeof names, cudaMemcpyDeviceToHost, st));
    DC3_CK(cudaStreamSynchronize(st));
    uint32_t *s12 = nullptr;  // the sample positions in rank order
    if (names < n02) {
        // equal triples: the reduced string's suffix array orders the samples
        sc.release(posA);
        sc.release(posB);
        uint32_t *sar = sc.get<uint32_t>(n02);
        if (!sar) return SA_ERR_NOMEM;
        int r = skew_gpu(NameLetters{red, n02}, n02, names, sar, st);
        if (r) return r;
        ranks_of_kernel<<<grid_of(n02), kThreads, 0, st>>>(sar, n02, red);
        DC3_CK(cudaGetLastError());
        s12 = sc.get<uint32_t>(n02);
        if (!s12) return SA_ERR_NOMEM;
        samples_in_order_kernel<<<grid_of(n02), kThreads, 0, st>>>(sar, n0, n02, s12);
        DC3_CK(cudaGetLastError());
        sc.release(sar);
    } else {
        // every name distinct: it is its sample's rank, and the triple order
        // is the rank order
        s12 = sorted;
        sc.release(other);
    }

    // Step 3: the mod-0 suffixes.
    uint32_t *cand = sc.get<uint32_t>(n02), *t0 = sc.get<uint32_t>(n0), *s0 = sc.get<uint32_t>(n0);
    uint8_t *flag = sc.get<uint8_t>(n02);
    uint64_t *d_cnt = sc.get<uint64_t>(1);
    uint32_t *k0 = sc.get<uint32_t>(n0), *k1 = sc.get<uint32_t>(n0);
    if (sc.failed) return SA_ERR_NOMEM;
    mod0_candidates_kernel<<<grid_of(n02), kThreads, 0, st>>>(s12, n02, cand, flag);
    DC3_CK(cudaGetLastError());
    {
        size_t tb = 0;
        DC3_CK(cub::DeviceSelect::Flagged(nullptr, tb, cand, flag, t0, d_cnt, n02, st));
        void *temp = sc.get<uint8_t>(tb);
        if (!temp) return SA_ERR_NOMEM;
        DC3_CK(cub::DeviceSelect::Flagged(temp, tb, cand, flag, t0, d_cnt, n02, st));
        sc.release(temp);
    }
    sc.release(cand);
    letter_key_kernel<<<grid_of(n0), kThreads, 0, st>>>(s, t0, n0, 0u, k0);
    DC3_CK(cudaGetLastError());
    cub::DoubleBuffer<uint32_t> kb0(k0, k1), pb0(t0, s0);
    int r = radix_by_key(kb0, pb0, n0, lb, st, sc);
    if (r) return r;
    const uint32_t *mod0 = pb0.Current();

    // Step 4: merge (the empty sample, rank 1, is dropped from the front).
    const uint64_t skip = (n0 > (n + 1) / 3) ? 1 : 0;
    sc.release(flag);
    sc.release(k0);
    sc.release(k1);
    uint4 *KA = sc.get<uint4>(n0), *KB = sc.get<uint4>(n02);
    if (sc.failed) return SA_ERR_NOMEM;
    const KeyOf<L> key{s, red, n, n0};
    merge_keys_kernel<<<grid_of(n0), kThreads, 0, st>>>(key, mod0, n0, KA);
    DC3_CK(cudaGetLastError());
    merge_keys_kernel<<<grid_of(n02 - skip), kThreads, 0, st>>>(key, s12 + skip, n02 - skip, KB);
    DC3_CK(cudaGetLastError());
    const uint64_t threads_of = (n + kMergeItems - 1) / kMergeItems;
    merge_kernel<<<grid_of(threads_of), kThreads, 0, st>>>(KA, mod0, n0, KB, s12 + skip, n02 - skip, sa);
    DC3_CK(cudaGetLastError());
    DC3_CK(cudaStreamSynchronize(st));
    return SA_OK;
}

}  // namespace

int build_suffix_array_dc3(sa_index *idx, cudaStream_t s) {
    const uint64_t n = idx->n;
    uint32_t *sa32 = nullptr;
    const bool narrow = idx->width == 4;
    if (narrow) {
        sa32 = reinterpret_cast<uint32_t *>(idx->sa);
    } else if (scratch_alloc(reinterpret_cast<void **>(&sa32), n * sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_NOMEM;
    }
    int r = skew_gpu(PackedLetters{idx->text, n}, n, 4u, sa32, s);
    if (r == SA_OK && !narrow) {
        widen_sa_kernel<<<grid_of(n), kThreads, 0, s>>>(sa32, n, reinterpret_cast<uint64_t *>(idx->sa));
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) r = status_from_cuda(e);
    }
    if (!narrow) scratch_free(sa32, s);
    return r;
}

}  // namespace sa
