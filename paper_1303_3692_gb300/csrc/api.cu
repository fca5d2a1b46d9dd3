// api.cu -- the extern "C" entry points declared in include/sa.h: argument
// checks, host/device staging, scratch memory and the index life cycle.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dc3.h"
#include "sa_internal.cuh"

namespace sa {

// An NVTX range over one library call on the calling host thread, so that
// profilers (ncu --nvtx, Nsight Systems) can select a call's kernels.  Costs a
// branch when no profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

int status_from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return SA_OK;
    if (e == cudaErrorMemoryAllocation) return SA_ERR_NOMEM;
    return SA_ERR_CUDA;
}

namespace {
std::mutex g_mu;
constexpr int kMaxDevices = 64;
cudaMemPool_t g_pool[kMaxDevices];
bool g_pool_ok[kMaxDevices];
int g_sms[kMaxDevices];
}  // namespace

// Library-private stream-ordered pool: scratch is allocated and released on
// the caller's stream; the pool keeps freed memory for reuse (trimmed after
// an index build, whose scratch is large).
cudaMemPool_t scratch_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    if (!g_pool_ok[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        if (cudaMemPoolCreate(&g_pool[dev], &props) != cudaSuccess) return nullptr;
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        g_pool_ok[dev] = true;
    }
    return g_pool[dev];
}

cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = scratch_pool(dev);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
}

void scratch_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int device_sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = v > 0 ? v : 1;
    }
    return g_sms[dev];
}

namespace {

bool on_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Scratch allocations released on the stream when the call returns.  Every
// block is returned 256-byte aligned (kernels read 32-byte records with one
// 256-bit load), whatever alignment the pool itself guarantees.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    bool failed = false;
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (failed) return nullptr;
        if (scratch_alloc(&p, count * sizeof(T) + 256 + 16, s) != cudaSuccess) {
            failed = true;
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        const uintptr_t a = ((uintptr_t)p + 255) & ~(uintptr_t)255;
        return reinterpret_cast<T *>(a);
    }
    ~Scratch() {
        for (void *p : ptrs) scratch_free(p, s);
    }
};

// Device copy of a caller buffer: the pointer itself if it is device memory,
// else a scratch copy filled on the stream.
template <typename T>
const T *device_view(const T *p, size_t count, Scratch &sc, cudaError_t *err) {
    if (p == nullptr || count == 0 || on_device(p)) return p;
    T *d = sc.get<T>(count);
    if (!d) {
        *err = cudaErrorMemoryAllocation;
        return nullptr;
    }
    cudaError_t e = cudaMemcpyAsync(d, p, count * sizeof(T), cudaMemcpyHostToDevice, sc.s);
    if (e != cudaSuccess) *err = e;
    return d;
}

uint32_t floor_log2(uint64_t x) {
    uint32_t l = 0;
    while (x > 1) {
        x >>= 1;
        l++;
    }
    return l;
}

constexpr uint32_t kDefaultDepth = 13;
// First-pass probes when the caller sets none.  With fewer suffixes than
// k-mers the entry's pivot settles most queries and two more probes settle
// nearly all; with more suffixes than k-mers (brackets of several suffixes and
// repeat copies) the first pass's warps would idle on their widest lanes, so
// every query the entry does not settle goes straight to the persistent pass.
// (Measured: 3 probes best at n/4^k = 0.37 and 0.72, 1 probe at 2.9.)
uint32_t default_front_probes(const sa_index *const *refs, uint32_t n_refs) {
    for (uint32_t r = 0; r < n_refs; r++) {
        const sa_index *x = refs[r];
        if (x->kmer_k && x->n > (1ull << (2 * x->kmer_k))) return 1;
    }
    return 3;
}
constexpr uint32_t kSmemBudget = 200 * 1024;

// Indexes of more device bytes than this (in one call) are searched in k-mer
// order: the random reads of a search over a larger footprint outrun the
// GPU's address-translation reach (measured on the GB300: 34-38 G random
// sectors/s up to 64 GB, 22 G/s at 80 GB, 8 G/s at 190 GB; 40 G/s when the
// reads in flight stay within a 1 GB slice of a 192 GB buffer).
// The order only narrows the reads in flight when the batch is much larger
// than the ~150,000 lanes the kernels keep busy at once.
constexpr uint64_t kKmerOrderMinBytes = 48ull << 30;
constexpr uint64_t kKmerOrderMinQueries = 1ull << 20;

// Whether a search of n_q queries over these indexes runs in k-mer order
// (order: the SA_PARAM_*_ORDER flags of the call).
bool use_kmer_order(const sa_index *const *refs, uint32_t n_refs, uint64_t n_q, uint32_t order) {
    uint64_t ktotal = 0, index_bytes = 0;
    for (uint32_t r = 0; r < n_refs; r++) {
        if (refs[r]->krt) ktotal += 1ull << (2 * refs[r]->kmer_k);
        index_bytes += refs[r]->device_bytes;
    }
    // (list slots are 32-bit: batches below 2^30 queries)
    if (ktotal == 0 || order == SA_PARAM_INPUT_ORDER || n_q >= (1ull << 30)) return false;
    return order == SA_PARAM_KMER_ORDER || (index_bytes > kKmerOrderMinBytes && n_q >= kKmerOrderMinQueries);
}

int check_refs(const sa_index *const *refs, uint32_t n_refs, uint32_t *width) {
    if (!refs || n_refs == 0 || n_refs > SA_MAX_REFS) return SA_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SA_ERR_CUDA;
    for (uint32_t r = 0; r < n_refs; r++) {
        if (!refs[r] || refs[r]->device != dev) return SA_ERR_ARG;
        if (r && refs[r]->width != refs[0]->width) return SA_ERR_ARG;
    }
    *width = refs[0]->width;
    return SA_OK;
}

// Per-index table depths for one call: each index's own depth, capped by the
// request, then the deepest tables are trimmed until all fit the budget.
uint32_t fill_ref_table(const sa_index *const *refs, uint32_t n_refs, uint32_t want_depth, RefTable *t,
                        uint32_t budget = kSmemBudget) {
    uint32_t use[SA_MAX_REFS];
    for (uint32_t r = 0; r < n_refs; r++) {
        use[r] = refs[r]->depth < want_depth ? refs[r]->depth : want_depth;
    }
    for (;;) {
        uint32_t total = 0, deepest = 0;
        for (uint32_t r = 0; r < n_refs; r++) {
            total += search_table_bytes(use[r]);
            if (use[r] > use[deepest]) deepest = r;
        }
        if (total <= budget || use[deepest] == 0) break;
        use[deepest]--;
    }
    uint32_t off = 0;
    uint64_t kbase = 0;
    for (uint32_t r = 0; r < n_refs; r++) {
        const sa_index *x = refs[r];
        RefDesc &d = t->r[r];
        d.kbase = kbase;
        if (x->krt) kbase += 1ull << (2 * x->kmer_k);
        d.text = x->text;
        d.sa = x->sa;
        d.keys = x->keys;
        d.keylen = x->keylen;
        d.rec = x->rec;
        d.krt = x->krt;
        d.kmer_k = x->kmer_k;
        d.n = x->n;
        d.depth = x->depth;
        d.use_depth = use[r];
        d.smem_off = off;
        off += search_table_bytes(use[r]);
    }
    return off;
}

// The search of a batch whose inputs are in device memory: ascii holds the
// batch's bases from offset `first` on (query q is ascii[q_off[q] - first ..
// q_off[q + 1] - first)), q_off and q_ref are device arrays and out device
// results.  Scratch comes from sc, on stream s.  *flags_out receives the
// call's device flags ([0] a byte that is not a base, [1] a wait that ran
// out, [3] a bad reference id).
int search_device(const sa_index *const *refs, uint32_t n_refs, uint32_t width, const char *ascii,
                  const uint64_t *q_off, const uint32_t *q_ref, uint64_t n_q, uint64_t first, uint64_t total,
                  sa_result *out, cudaStream_t s, const sa_search_params *params, bool plain, uint32_t trunc_cap,
                  Scratch &sc, int **flags_out, uint64_t *tile_kept = nullptr) {
    const uint32_t order = params ? params->flags & (SA_PARAM_KMER_ORDER | SA_PARAM_INPUT_ORDER) : 0u;
    if (order == (SA_PARAM_KMER_ORDER | SA_PARAM_INPUT_ORDER)) return SA_ERR_ARG;
    const uint32_t threads = params && params->threads_per_block ? params->threads_per_block : 1024;
    uint32_t bps = params && params->blocks_per_sm ? params->blocks_per_sm : 1;
    if (threads < 32 || threads > 1024 || threads % 32 || bps == 0 || threads * bps > 2048) return SA_ERR_ARG;
    if (threads * bps > 1024) bps = 1024 / threads;  // the persistent kernel takes 64 registers a thread
    if (params && params->front_probes > 64) return SA_ERR_ARG;
    const bool strand_bits = params && (params->flags & SA_PARAM_STRAND_PER_QUERY);
    const bool revcomp = params && (params->flags & SA_PARAM_REVERSE_COMPLEMENT);
    if (strand_bits && (revcomp || !q_ref)) return SA_ERR_ARG;
    cudaError_t err = cudaSuccess;
    const uint64_t nwords = (total + 31) / 32;
    // both packings, one after the other, when each query names its strand
    const uint64_t tq_words = (nwords + SA_TQ_PAD_WORDS) * (strand_bits ? 2 : 1);
    // list and worklist records hold a query's first base in 48 bits (a batch
    // that large could not be resident anyway)
    if (!plain && tq_words * 32 >= kListMaxBase) return SA_ERR_ARG;
    uint64_t *tq = sc.get<uint64_t>(tq_words);
    uint32_t *tv = sc.get<uint32_t>(tq_words);
    uint4 *wrec = plain ? nullptr : sc.get<uint4>(4 * n_q);
    uint64_t ktotal = 0;
    for (uint32_t r = 0; r < n_refs; r++)
        if (refs[r]->krt) ktotal += 1ull << (2 * refs[r]->kmer_k);
    const bool kmer_order = !plain && use_kmer_order(refs, n_refs, n_q, order);
    uint4 *wrec_in = kmer_order ? sc.get<uint4>(4 * list_capacity(n_q)) : nullptr;
    uint32_t *bplan = kmer_order ? sc.get<uint32_t>(kPlanWords) : nullptr;
    // [0] pack error, [1] status, [2] worklist count, [3] bad reference id,
    // [4] records of the k-mer-ordered list, [5] a non-base byte in the batch
    int *flags = sc.get<int>(8);
    unsigned long long *counter = sc.get<unsigned long long>(1);
    if (sc.failed) return SA_ERR_NOMEM;
    if (((uintptr_t)wrec & 31u) != 0) return SA_ERR_CUDA;  // the search reads 32-byte records
    if ((err = cudaMemsetAsync(flags, 0, 8 * sizeof(int), s)) != cudaSuccess) return status_from_cuda(err);
    if ((err = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return status_from_cuda(err);
    if (bplan && (err = cudaMemsetAsync(bplan, 0, kPlanWords * sizeof(uint32_t), s)) != cudaSuccess)
        return status_from_cuda(err);
    *flags_out = flags;

    SearchLaunch L;
    memset(&L, 0, sizeof L);
    // shared memory per SM is 228 KB; each CTA also holds ~4 KB of descriptors
    const uint32_t per_cta = 224u * 1024u / bps - 6144u;
    const uint32_t budget = per_cta < kSmemBudget ? per_cta : kSmemBudget;
    const uint32_t want_depth = params && params->key_depth ? params->key_depth : kDefaultDepth;
    L.smem_bytes = fill_ref_table(refs, n_refs, plain ? 0 : want_depth, &L.refs, budget);
    L.n_refs = n_refs;
    L.width = width;
    L.ascii = ascii;
    L.tq = tq;
    L.tv = tv;
    L.nwords = nwords;
    L.q_off = q_off;
    L.first = first;
    L.total = total;
    L.q_ref = q_ref;
    L.n_q = n_q;
    L.wrec = wrec;
    L.wl_count = reinterpret_cast<uint32_t *>(flags + 2);
    L.out = out;
    L.pack_err = flags;
    L.counter = counter;
    L.status = flags + 1;
    const int sms = device_sm_count();
    L.threads = threads;
    L.blocks = (uint32_t)sms * bps;
    L.chunk = params && params->chunk ? params->chunk : 64;
    // with the queries in k-mer order neighbouring lanes share pages and rows,
    // and the first pass does best with three probes (measured)
    L.front_probes = params && params->front_probes ? params->front_probes
                                                    : (kmer_order ? 3u : default_front_probes(refs, n_refs));
    L.revcomp = revcomp;
    L.strand_bits = strand_bits;
    L.rc_base = strand_bits ? (nwords + SA_TQ_PAD_WORDS) * 32 : 0;
    L.expire_waits = params && (params->flags & SA_PARAM_EXPIRE_WAITS);
    L.trunc_cap = trunc_cap;
    L.tile_kept = tile_kept;
    L.tile_sum_by_warp = !kmer_order;
    L.ktotal = ktotal;
    L.bplan = bplan;
    L.wrec_in = wrec_in;
    L.wl_in_count = reinterpret_cast<uint32_t *>(flags + 4);
    L.bad_ref = flags + 3;
    L.batch_dirty = flags + 5;

    if ((err = launch_pack_batch(L, tq, tv, s)) != cudaSuccess) return status_from_cuda(err);
    cudaEvent_t ev0 = params ? reinterpret_cast<cudaEvent_t>(params->search_events[0]) : nullptr;
    cudaEvent_t ev1 = params ? reinterpret_cast<cudaEvent_t>(params->search_events[1]) : nullptr;
    if (ev0 && (err = cudaEventRecord(ev0, s)) != cudaSuccess) return status_from_cuda(err);
    if (plain) {
        err = launch_search_plain(L, s);
    } else {
        if (kmer_order) err = launch_bucketed_worklist(L, wrec_in, s);
        if (err == cudaSuccess) err = launch_front(L, s);
        if (err == cudaSuccess) err = launch_search(L, s);
    }
    if (err != cudaSuccess) return status_from_cuda(err);
    if (ev1 && (err = cudaEventRecord(ev1, s)) != cudaSuccess) return status_from_cuda(err);
    return SA_OK;
}

// The call's status from its device flags read back to the host.
int host_status(const int hflags[4]) {
    if (hflags[1]) return hflags[1];
    if (hflags[0]) return SA_ERR_BASE;
    if (hflags[3]) return SA_ERR_ARG;
    return SA_OK;
}

int search_impl(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                const uint32_t *q_ref, uint64_t n_q, sa_result *out, void *stream, const sa_search_params *params,
                bool plain, uint32_t trunc_cap = ~0u, uint64_t *tile_kept = nullptr) {
    NvtxRange range(plain ? "sa_search_plain" : "sa_search");
    uint32_t width = 0;
    int st = check_refs(refs, n_refs, &width);
    if (st) return st;
    if (n_q == 0) return SA_OK;
    if (!q_offsets || !out || (n_refs > 1 && !q_ref) || n_q >= (1ull << 32)) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // First and last offset: given, read directly, or with one small synchronous copy.
    uint64_t first = 0, last = 0;
    const bool off_dev = on_device(q_offsets);
    if (params && (params->flags & SA_PARAM_Q_RANGE)) {
        first = params->q_first;
        last = params->q_first + params->q_total;
    } else if (off_dev) {
        uint64_t fl[2];
        cudaError_t e = cudaMemcpyAsync(&fl[0], q_offsets, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&fl[1], q_offsets + n_q, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return status_from_cuda(e);
        first = fl[0];
        last = fl[1];
    } else {
        first = q_offsets[0];
        last = q_offsets[n_q];
    }
    if (last < first) return SA_ERR_ARG;
    const uint64_t total = last - first;
    if (total > 0 && !q_bases) return SA_ERR_ARG;
    const bool out_dev = on_device(out);
    if (out_dev && ((uintptr_t)out & 31u)) return SA_ERR_ARG;  // results are stored as whole 32-byte sectors
    int *dstatus = params ? params->device_status : nullptr;
    if (dstatus && !on_device(dstatus)) return SA_ERR_ARG;

    Scratch sc{s};
    cudaError_t err = cudaSuccess;
    const char *bases_d = nullptr;
    if (total > 0) {
        if (on_device(q_bases)) {
            bases_d = q_bases + first;
        } else {
            char *d = sc.get<char>(total);
            if (!d) return SA_ERR_NOMEM;
            err = cudaMemcpyAsync(d, q_bases + first, total, cudaMemcpyHostToDevice, s);
            bases_d = d;
        }
    }
    const uint64_t *off_d = device_view(q_offsets, n_q + 1, sc, &err);
    const uint32_t *ref_d = n_refs > 1 || q_ref ? device_view(q_ref, n_q, sc, &err) : nullptr;
    sa_result *out_d = out_dev ? out : sc.get<sa_result>(n_q);
    if (sc.failed) return SA_ERR_NOMEM;
    if (err != cudaSuccess) return status_from_cuda(err);
    int *flags = nullptr;
    st = search_device(refs, n_refs, width, bases_d, off_d, ref_d, n_q, first, total, out_d, s, params, plain,
                       trunc_cap, sc, &flags, tile_kept);
    if (st) return st;
    if (dstatus && (err = launch_search_status(flags, dstatus, s)) != cudaSuccess) return status_from_cuda(err);
    if (!out_dev) {
        int hflags[4] = {0, 0, 0, 0};
        if ((err = cudaMemcpyAsync(out, out_d, n_q * sizeof(sa_result), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        if ((err = cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return status_from_cuda(err);
        return host_status(hflags);
    }
    return SA_OK;
}

void free_index(sa_index *idx) {
    if (!idx) return;
    if (idx->text) cudaFree(idx->text);
    if (idx->sa) cudaFree(idx->sa);
    if (idx->keys) cudaFree(idx->keys);
    if (idx->keylen) cudaFree(idx->keylen);
    if (idx->rec) cudaFree(idx->rec);
    if (idx->krt) cudaFree(idx->krt);
    delete idx;
}

uint32_t table_entries(uint32_t depth) { return depth >= 4 ? (1u << depth) : 16u; }

// Automatic k: the largest k with 4^k <= 3n, in 1..15 (at least one k-mer
// entry per three suffixes on average, so that most brackets hold one or
// two suffixes; the table takes at most 192 bytes per base).
uint32_t auto_kmer_k(uint64_t n) {
    uint32_t k = 1;
    while (k < 15 && (1ull << (2 * (k + 1))) <= 3 * n) k++;
    return k;
}

// Allocates the device arrays of an index whose n, width, depth and kmer_k
// are set: first the text, suffix array and key table; the records (32n
// bytes) and the k-mer table (64 * 4^k bytes) are allocated separately,
// after the build's scratch has been returned, so the two never coexist.
int alloc_index(sa_index *idx) {
    idx->nwords = (idx->n + 31) / 32;
    const size_t tb = (idx->nwords + SA_PAD_WORDS) * sizeof(uint64_t);
    const size_t sb = idx->n * (size_t)idx->width;
    const size_t kb = table_entries(idx->depth) * sizeof(uint4);
    const size_t lb = table_entries(idx->depth);
    if (cudaMalloc(&idx->text, tb) != cudaSuccess || cudaMalloc(&idx->sa, sb) != cudaSuccess ||
        cudaMalloc(&idx->keys, kb) != cudaSuccess || cudaMalloc(&idx->keylen, lb) != cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_NOMEM;
    }
    idx->device_bytes = tb + sb + kb + lb;
    return SA_OK;
}

int alloc_search_arrays(sa_index *idx) {
    const size_t rb = idx->n * 2 * sizeof(uint4);
    if (cudaMalloc(&idx->rec, rb) != cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_NOMEM;
    }
    size_t mb = 0;
    if (idx->kmer_k) {
        mb = (1ull << (2 * idx->kmer_k)) * 4 * sizeof(uint4);
        if (cudaMalloc(&idx->krt, mb) != cudaSuccess) {
            cudaGetLastError();
            return SA_ERR_NOMEM;
        }
    }
    idx->device_bytes += rb + mb;
    return SA_OK;
}

uint64_t fnv1a(uint64_t h, const void *p, size_t bytes) {
    const uint8_t *b = reinterpret_cast<const uint8_t *>(p);
    for (size_t i = 0; i < bytes; i++) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct FileHeader {
    char magic[8];
    uint32_t version, width;
    uint64_t n;
    uint32_t depth, kmer_k;
    uint64_t nwords;
    uint64_t checksum;
};

const char kMagic[8] = {'S', 'A', 'G', 'B', '3', '0', '0', '\0'};

}  // namespace
}  // namespace sa

namespace sa {
// Host batches of at least this many queries (bases and offsets in host
// memory) run in chunks on two library streams: each chunk's upload overlaps
// the previous chunk's kernels and the one before's downloads, instead of one
// upload of the whole batch, then the kernels, then the downloads.
constexpr uint64_t kPipelineMinQueries = 1ull << 21;
int search_pipelined(const sa_index *const *refs, uint32_t n_refs, uint32_t width, const char *q_bases,
                     const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q, sa_result *out,
                     cudaStream_t s, const sa_search_params *params, bool locate, uint32_t cap,
                     uint64_t *out_offsets, void *out_pos, uint64_t capacity);
}  // namespace sa

using namespace sa;

extern "C" {

int sa_build(const char *text, uint64_t n, uint32_t flags, void *stream, sa_index **out) {
    NvtxRange range("sa_build");
    if (!out) return SA_ERR_ARG;
    *out = nullptr;
    if (!text || n == 0 || n >= 0xFFFFFFFFull) return SA_ERR_ARG;
    const uint32_t wflags = flags & (SA_W32 | SA_W64);
    if (wflags != SA_W32 && wflags != SA_W64) return SA_ERR_ARG;
    if (flags & ~(SA_W32 | SA_W64 | SA_NO_KMER | SA_BUILD_HOST | SA_BUILD_DC3 | SA_KMER_K(15))) return SA_ERR_ARG;
    if ((flags & SA_BUILD_HOST) && (flags & SA_BUILD_DC3)) return SA_ERR_ARG;
    const uint32_t want_k = (flags >> 8) & 15u;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    sa_index *idx = new (std::nothrow) sa_index();
    if (!idx) return SA_ERR_NOMEM;
    if (cudaGetDevice(&idx->device) != cudaSuccess) {
        delete idx;
        return SA_ERR_CUDA;
    }
    idx->n = n;
    idx->width = wflags == SA_W32 ? 4 : 8;
    const uint32_t lg = floor_log2(n);
    idx->depth = lg < kDefaultDepth ? lg : kDefaultDepth;
    idx->kmer_k = (flags & SA_NO_KMER) ? 0u : (want_k ? want_k : auto_kmer_k(n));
    int st = alloc_index(idx);
    if (st) {
        free_index(idx);
        return st;
    }
    {
        Scratch sc{s};
        cudaError_t err = cudaSuccess;
        const char *text_d = device_view(text, n, sc, &err);
        int *flag = sc.get<int>(1);
        if (sc.failed) {
            free_index(idx);
            return SA_ERR_NOMEM;
        }
        int hflag = 0;
        if (err == cudaSuccess) err = cudaMemsetAsync(flag, 0, sizeof(int), s);
        if (err == cudaSuccess) err = launch_pack_text(text_d, n, idx->text, idx->nwords + SA_PAD_WORDS, flag, s);
        if (err == cudaSuccess) err = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) {
            free_index(idx);
            return status_from_cuda(err);
        }
        if (hflag) {
            free_index(idx);
            return SA_ERR_BASE;
        }
    }
    if (flags & SA_BUILD_HOST) {
        std::vector<char> copy;
        const char *host_text = text;
        if (on_device(text)) {
            try {
                copy.resize(n);
            } catch (const std::bad_alloc &) {
                free_index(idx);
                return SA_ERR_NOMEM;
            }
            cudaError_t err = cudaMemcpyAsync(copy.data(), text, n, cudaMemcpyDeviceToHost, s);
            if (err == cudaSuccess) err = cudaStreamSynchronize(s);
            if (err != cudaSuccess) {
                free_index(idx);
                return status_from_cuda(err);
            }
            host_text = copy.data();
        }
        st = build_suffix_array_host(idx, host_text, stream);
    } else if (flags & SA_BUILD_DC3) {
        st = build_suffix_array_dc3(idx, s);
    } else {
        st = build_suffix_array(idx, s);
    }
    cudaStreamSynchronize(s);
    cudaMemPoolTrimTo(scratch_pool(idx->device), 0);
    if (st == SA_OK) st = alloc_search_arrays(idx);
    if (st == SA_OK) {
        cudaError_t err = launch_build_keys(idx, s);
        if (err == cudaSuccess) err = launch_build_records(idx, s);
        if (err == cudaSuccess) err = launch_build_kmer(idx, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        cudaMemPoolTrimTo(scratch_pool(idx->device), 0);
        st = status_from_cuda(err);
    }
    if (st) {
        free_index(idx);
        return st;
    }
    *out = idx;
    return SA_OK;
}

}  // extern "C"

namespace sa {
// Whether a call takes the chunked host path: bases and offsets in host
// memory and a large batch.
bool pipelined(const char *q_bases, const uint64_t *q_offsets, uint64_t n_q) {
    return n_q >= kPipelineMinQueries && q_offsets && !on_device(q_offsets) && (!q_bases || !on_device(q_bases));
}

int search_pipelined_entry(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                           const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q, sa_result *out,
                           void *stream, const sa_search_params *params, bool locate, uint32_t cap,
                           uint64_t *out_offsets, void *out_pos, uint64_t capacity) {
    NvtxRange range(locate ? "sa_search_locate" : "sa_search");
    uint32_t width = 0;
    int st = check_refs(refs, n_refs, &width);
    if (st) return st;
    if (!out || (n_refs > 1 && !q_ref) || n_q >= (1ull << 32) || (locate && !out_offsets)) return SA_ERR_ARG;
    return search_pipelined(refs, n_refs, width, q_bases, q_offsets, q_ref, n_q, out,
                            reinterpret_cast<cudaStream_t>(stream), params, locate, cap, out_offsets, out_pos,
                            capacity);
}
}  // namespace sa

extern "C" {

int sa_search_batch(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                    const uint32_t *q_ref, uint64_t n_q, sa_result *out, void *stream) {
    if (sa::pipelined(q_bases, q_offsets, n_q))
        return sa::search_pipelined_entry(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, nullptr, false,
                                          0, nullptr, nullptr, 0);
    return search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, nullptr, false);
}

int sa_search_batch_ex(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                       const uint32_t *q_ref, uint64_t n_q, sa_result *out, void *stream,
                       const sa_search_params *params) {
    if (sa::pipelined(q_bases, q_offsets, n_q))
        return sa::search_pipelined_entry(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, params, false,
                                          0, nullptr, nullptr, 0);
    return search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, params, false);
}

int sa_search_batch_plain(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                          const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q, sa_result *out,
                          void *stream) {
    return search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, nullptr, true);
}

}  // extern "C"

namespace sa {

// Locate on device-resident inputs and outputs; base_in (device, or null for
// 0) is added to every offset, for one chunk of a larger batch.
int locate_device(const sa_index *const *refs, uint32_t n_refs, uint32_t width, const uint32_t *ref_d,
                  const sa_result *res_d, uint64_t n_q, uint32_t cap, uint64_t *off_d, void *pos_d,
                  uint64_t capacity, const uint64_t *base_in, int *overflow, cudaStream_t s, Scratch &sc,
                  uint64_t *presummed = nullptr) {
    // presummed: the tile sums, already added up by the search kernels
    uint64_t *partials = presummed ? presummed : sc.get<uint64_t>(locate_tiles(n_q) + 1);
    if (sc.failed) return SA_ERR_NOMEM;
    LocateLaunch L;
    memset(&L, 0, sizeof L);
    fill_ref_table(refs, n_refs, 0, &L.refs);
    L.n_refs = n_refs;
    L.width = width;
    L.q_ref = ref_d;
    L.res = res_d;
    L.n_q = n_q;
    L.cap = cap;
    L.out_offsets = off_d;
    L.out_pos = pos_d;
    L.capacity = pos_d ? capacity : 0;
    L.partials = partials;
    L.presummed = presummed != nullptr;
    L.overflow = overflow;
    L.base_in = base_in;
    return status_from_cuda(launch_locate(L, s));
}

int locate_impl(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref, const sa_result *res,
                uint64_t n_q, uint32_t cap, uint64_t *out_offsets, void *out_pos, uint64_t out_pos_capacity,
                void *stream, int *dstatus = nullptr, uint64_t *presummed = nullptr) {
    NvtxRange range("sa_locate");
    uint32_t width = 0;
    int st = check_refs(refs, n_refs, &width);
    if (st) return st;
    if (!out_offsets || (n_q && !res) || (n_refs > 1 && n_q && !q_ref)) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc{s};
    cudaError_t err = cudaSuccess;
    const sa_result *res_d = device_view(res, n_q, sc, &err);
    const uint32_t *ref_d = q_ref ? device_view(q_ref, n_q, sc, &err) : nullptr;
    const bool off_dev = on_device(out_offsets);
    uint64_t *off_d = off_dev ? out_offsets : sc.get<uint64_t>(n_q + 1);
    const bool pos_dev = out_pos == nullptr || on_device(out_pos);
    void *pos_d = out_pos;
    if (!pos_dev && out_pos_capacity) pos_d = sc.get<uint8_t>(out_pos_capacity * width);
    if (!pos_dev && !out_pos_capacity) pos_d = nullptr;
    int *overflow = dstatus && pos_d ? sc.get<int>(1) : nullptr;
    if (sc.failed) return SA_ERR_NOMEM;
    if (err != cudaSuccess) return status_from_cuda(err);
    if (overflow && (err = cudaMemsetAsync(overflow, 0, sizeof(int), s)) != cudaSuccess) return status_from_cuda(err);
    st = locate_device(refs, n_refs, width, ref_d, res_d, n_q, cap, off_d, pos_d, out_pos_capacity, nullptr, overflow,
                       s, sc, presummed);
    if (st) return st;
    if (overflow && (err = launch_capacity_status(overflow, dstatus, s)) != cudaSuccess) return status_from_cuda(err);
    if (!off_dev || !pos_dev) {
        uint64_t total = 0;
        if ((err = cudaMemcpyAsync(&total, off_d + n_q, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return status_from_cuda(err);
        if (!off_dev &&
            (err = cudaMemcpyAsync(out_offsets, off_d, (n_q + 1) * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        const uint64_t kept = total < out_pos_capacity ? total : out_pos_capacity;
        if (!pos_dev && pos_d && kept &&
            (err = cudaMemcpyAsync(out_pos, pos_d, kept * width, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return status_from_cuda(err);
        if (out_pos && total > out_pos_capacity) return SA_ERR_CAPACITY;
    }
    return SA_OK;
}

constexpr int kPipelineStreams = 2;

cudaError_t pipeline_streams(cudaStream_t out[kPipelineStreams]) {
    static std::mutex mu;
    static cudaStream_t st[kMaxDevices][kPipelineStreams];
    static bool ok[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!ok[dev]) {
        for (int i = 0; i < kPipelineStreams; i++)
            if ((e = cudaStreamCreateWithFlags(&st[dev][i], cudaStreamNonBlocking)) != cudaSuccess) return e;
        ok[dev] = true;
    }
    for (int i = 0; i < kPipelineStreams; i++) out[i] = st[dev][i];
    return cudaSuccess;
}

// Events of one pipelined call, destroyed when it returns (after the streams
// that use them have been waited for, or are ordered before the caller's).
struct Events {
    std::vector<cudaEvent_t> ev;
    cudaEvent_t make() {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ev.push_back(e);
        return e;
    }
    ~Events() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

// sa_search_batch / sa_search_locate with q_bases and q_offsets in host
// memory, in chunks of queries (see kPipelineMinQueries).  Same results,
// status and synchronization as the unchunked calls.
int search_pipelined(const sa_index *const *refs, uint32_t n_refs, uint32_t width, const char *q_bases,
                     const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q, sa_result *out,
                     cudaStream_t s, const sa_search_params *params, bool locate, uint32_t cap,
                     uint64_t *out_offsets, void *out_pos, uint64_t capacity) {
    // Chunks of about n_q / 12 queries (at least 2^20); the last such chunk's
    // queries go in four quarter chunks, so that less work is left after the
    // final upload.
    const uint64_t per = (n_q + 11) / 12 > (1ull << 20) ? (n_q + 11) / 12 : (1ull << 20);
    std::vector<uint64_t> cut;  // chunk c is [cut[c], cut[c + 1])
    try {
        cut.push_back(0);
        while (n_q - cut.back() > per) cut.push_back(cut.back() + per);
        const uint64_t rest = n_q - cut.back(), quarter = (rest + 3) / 4;
        for (int j = 0; j < 4 && cut.back() < n_q; j++) cut.push_back(cut.back() + quarter < n_q ? cut.back() + quarter : n_q);
    } catch (const std::bad_alloc &) {
        return SA_ERR_NOMEM;
    }
    const uint64_t n_chunks = cut.size() - 1;
    uint64_t max_bases = 0;
    for (uint64_t c = 0; c < n_chunks; c++) {
        const uint64_t a = cut[c], b = cut[c + 1];
        if (q_offsets[b] < q_offsets[a]) return SA_ERR_ARG;
        if (q_offsets[b] - q_offsets[a] > max_bases) max_bases = q_offsets[b] - q_offsets[a];
    }
    if (max_bases > 0 && !q_bases) return SA_ERR_ARG;
    const bool out_dev = on_device(out);
    if (out_dev && ((uintptr_t)out & 31u)) return SA_ERR_ARG;
    const bool ref_dev = q_ref && on_device(q_ref);
    const bool off_dev = !locate || on_device(out_offsets);
    const bool pos_dev = !locate || out_pos == nullptr || on_device(out_pos);
    // A host positions array the device can address (pinned or registered)
    // receives each chunk's positions as soon as its locate is done, instead
    // of all of them after the last chunk.
    void *pos_host_dev = nullptr;
    if (!pos_dev && capacity) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, out_pos) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer != nullptr)
            pos_host_dev = pa.devicePointer;
        else
            cudaGetLastError();
    }
    int *dstatus = params ? params->device_status : nullptr;
    if (dstatus && !on_device(dstatus)) return SA_ERR_ARG;
    sa_search_params cp;  // the caller's knobs, without the per-call extras the chunks do not take
    memset(&cp, 0, sizeof cp);
    if (params) cp = *params;
    cp.search_events[0] = cp.search_events[1] = nullptr;
    cp.device_status = nullptr;
    cp.flags &= ~SA_PARAM_Q_RANGE;
    // the order is decided for the whole batch, not per chunk
    const uint32_t order = cp.flags & (SA_PARAM_KMER_ORDER | SA_PARAM_INPUT_ORDER);
    if (order == (SA_PARAM_KMER_ORDER | SA_PARAM_INPUT_ORDER)) return SA_ERR_ARG;
    if (use_kmer_order(refs, n_refs, n_q, order)) cp.flags = (cp.flags & ~SA_PARAM_INPUT_ORDER) | SA_PARAM_KMER_ORDER;

    cudaStream_t ts[kPipelineStreams];
    cudaError_t err = pipeline_streams(ts);
    if (err != cudaSuccess) return status_from_cuda(err);
    Events evs;
    int st = SA_OK;
    uint64_t total = 0;
    int hstat[2] = {0, 0};
    {
        Scratch sc{s};
        sa_result *out_d = out_dev ? out : sc.get<sa_result>(n_q);
        uint64_t *off_d = off_dev ? out_offsets : sc.get<uint64_t>(n_q + 1);
        void *pos_d = pos_dev ? out_pos : (capacity ? sc.get<uint8_t>(capacity * width) : nullptr);
        char *slot_bases[kPipelineStreams];
        uint64_t *slot_off[kPipelineStreams];
        uint32_t *slot_ref[kPipelineStreams];
        for (int i = 0; i < kPipelineStreams; i++) {
            slot_bases[i] = sc.get<char>(max_bases);
            slot_off[i] = sc.get<uint64_t>(per + 1);
            slot_ref[i] = q_ref && !ref_dev ? sc.get<uint32_t>(per) : nullptr;
        }
        // [0] the chunks' statuses folded (the highest precedence seen), [1]
        // capacity overflow, then a zero base for the first chunk's offsets
        int *stat_d = sc.get<int>(4);
        if (sc.failed) return SA_ERR_NOMEM;
        const uint64_t *zero = reinterpret_cast<const uint64_t *>(stat_d + 2);
        if ((err = cudaMemsetAsync(stat_d, 0, 4 * sizeof(int), s)) != cudaSuccess) return status_from_cuda(err);
        cudaEvent_t start = evs.make(), loc_done[kPipelineStreams], fin[kPipelineStreams];
        for (int i = 0; i < kPipelineStreams; i++) {
            loc_done[i] = evs.make();
            fin[i] = evs.make();
        }
        if (!start || evs.ev.size() != 1 + 2 * kPipelineStreams) return SA_ERR_CUDA;
        if ((err = cudaEventRecord(start, s)) != cudaSuccess) return status_from_cuda(err);
        for (int i = 0; i < kPipelineStreams; i++)
            if ((err = cudaStreamWaitEvent(ts[i], start, 0)) != cudaSuccess) return status_from_cuda(err);
        for (uint64_t c = 0; c < n_chunks && st == SA_OK; c++) {
            const int i = (int)(c % kPipelineStreams);
            cudaStream_t t = ts[i];
            const uint64_t a = cut[c], b = cut[c + 1], nq = b - a;
            const uint64_t ba = q_offsets[a], nb = q_offsets[b] - ba;
            if (nb && (err = cudaMemcpyAsync(slot_bases[i], q_bases + ba, nb, cudaMemcpyHostToDevice, t)) != cudaSuccess)
                break;
            if ((err = cudaMemcpyAsync(slot_off[i], q_offsets + a, (nq + 1) * 8, cudaMemcpyHostToDevice, t)) !=
                cudaSuccess)
                break;
            const uint32_t *ref_c = q_ref ? (ref_dev ? q_ref + a : slot_ref[i]) : nullptr;
            if (q_ref && !ref_dev &&
                (err = cudaMemcpyAsync(slot_ref[i], q_ref + a, nq * 4, cudaMemcpyHostToDevice, t)) != cudaSuccess)
                break;
            Scratch csc{t};
            int *flags = nullptr;
            st = search_device(refs, n_refs, width, slot_bases[i], slot_off[i], ref_c, nq, ba, nb, out_d + a, t, &cp,
                               false, locate ? cap : ~0u, csc, &flags);
            if (st) break;
            if ((err = launch_fold_status(flags, stat_d, t)) != cudaSuccess) break;
            if (locate) {
                if (c > 0 && (err = cudaStreamWaitEvent(t, loc_done[(c - 1) % kPipelineStreams], 0)) != cudaSuccess)
                    break;
                st = locate_device(refs, n_refs, width, ref_c, out_d + a, nq, cap, off_d + a, pos_d, capacity,
                                   c ? off_d + a : zero, stat_d + 1, t, csc);
                if (st) break;
                if ((err = cudaEventRecord(loc_done[i], t)) != cudaSuccess) break;
                if (pos_host_dev && (err = launch_copy_positions(off_d + a, off_d + b, pos_d, pos_host_dev, width,
                                                                 capacity, t)) != cudaSuccess)
                    break;
                if (!off_dev && (err = cudaMemcpyAsync(out_offsets + a, off_d + a, nq * 8, cudaMemcpyDeviceToHost,
                                                       t)) != cudaSuccess)
                    break;
            }
            if (!out_dev && (err = cudaMemcpyAsync(out + a, out_d + a, nq * sizeof(sa_result), cudaMemcpyDeviceToHost,
                                                   t)) != cudaSuccess)
                break;
        }
        // join the library streams into the caller's
        for (int i = 0; i < kPipelineStreams; i++) {
            cudaError_t e = cudaEventRecord(fin[i], ts[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fin[i], 0);
            if (e != cudaSuccess && err == cudaSuccess) err = e;
        }
        if (st) return st;
        if (err != cudaSuccess) return status_from_cuda(err);
        if (dstatus && (err = launch_fold_final(stat_d, locate && pos_d, dstatus, s)) != cudaSuccess)
            return status_from_cuda(err);
        const bool host_out = !out_dev || !off_dev || !pos_dev;
        if (host_out) {
            if (locate && (err = cudaMemcpyAsync(&total, off_d + n_q, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return status_from_cuda(err);
            if ((err = cudaMemcpyAsync(hstat, stat_d, sizeof hstat, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return status_from_cuda(err);
            if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return status_from_cuda(err);
            if (locate && !off_dev) out_offsets[n_q] = total;
            const uint64_t kept = total < capacity ? total : capacity;
            if (locate && !pos_dev && pos_d && kept && !pos_host_dev) {
                if ((err = cudaMemcpyAsync(out_pos, pos_d, kept * width, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                    return status_from_cuda(err);
                if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return status_from_cuda(err);
            }
        }
        if (!host_out) return SA_OK;
    }
    if (hstat[0]) return hstat[0] == 3 ? SA_ERR_TIMEOUT : hstat[0] == 2 ? SA_ERR_BASE : SA_ERR_ARG;
    if (locate && out_pos && total > capacity) return SA_ERR_CAPACITY;
    return SA_OK;
}

}  // namespace sa

extern "C" {

int sa_locate(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref, const sa_result *res,
              uint64_t n_q, uint32_t cap, uint64_t *out_offsets, void *out_pos, uint64_t out_pos_capacity,
              void *stream) {
    return sa::locate_impl(refs, n_refs, q_ref, res, n_q, cap, out_offsets, out_pos, out_pos_capacity, stream);
}

int sa_search_locate(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                     const uint32_t *q_ref, uint64_t n_q, sa_result *out, uint32_t cap, uint64_t *out_offsets,
                     void *out_pos, uint64_t out_pos_capacity, void *stream, const sa_search_params *params) {
    using namespace sa;
    if (!out_offsets || (n_q && !out)) return SA_ERR_ARG;
    if (pipelined(q_bases, q_offsets, n_q))
        return search_pipelined_entry(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, params, true, cap,
                                      out_offsets, out_pos, out_pos_capacity);
    NvtxRange range("sa_search_locate");
    // the locate's tile sums, added up by the search kernels as they store
    // each result (so the locate need not read every result for them)
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Scratch sc{s};
    uint64_t *tile_kept = sc.get<uint64_t>(locate_tiles(n_q) + 1);
    if (sc.failed) return SA_ERR_NOMEM;
    cudaError_t err = cudaMemsetAsync(tile_kept, 0, (locate_tiles(n_q) + 1) * sizeof(uint64_t), s);
    if (err != cudaSuccess) return status_from_cuda(err);
    const int st = search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, params, false, cap,
                               tile_kept);
    if (st && st != SA_ERR_BASE && st != SA_ERR_ARG) return st;
    // invalid queries carry the all-ones result (no positions); the rest are located
    int *dstatus = params ? params->device_status : nullptr;
    const int lst = locate_impl(refs, n_refs, q_ref, out, n_q, cap, out_offsets, out_pos, out_pos_capacity, stream,
                                dstatus, st == SA_OK ? tile_kept : nullptr);
    return lst ? lst : st;
}

// sa_locate without allocation: device buffers only, scan scratch in the
// static array of locate.cu (see include/sa.h for who needs this and why).
int sa_locate_noalloc(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref, const sa_result *res,
                      uint64_t n_q, uint32_t cap, uint64_t *out_offsets, void *out_pos, uint64_t out_pos_capacity,
                      void *stream) {
    NvtxRange range("sa_locate_noalloc");
    if (n_q > SA_LOCATE_NOALLOC_MAX_QUERIES) return SA_ERR_CAPACITY;
    uint32_t width = 0;
    int st = check_refs(refs, n_refs, &width);
    if (st) return st;
    if (!out_offsets || (n_q && !res) || (n_refs > 1 && n_q && !q_ref)) return SA_ERR_ARG;
    if (!on_device(out_offsets) || (n_q && !on_device(res)) || (q_ref && !on_device(q_ref)) ||
        (out_pos && !on_device(out_pos)))
        return SA_ERR_ARG;
    uint64_t *partials = nullptr, entries = 0;
    cudaError_t err = locate_static_partials(&partials, &entries);
    if (err != cudaSuccess) return status_from_cuda(err);
    if (locate_tiles(n_q) + 1 > entries) return SA_ERR_CAPACITY;
    LocateLaunch L;
    memset(&L, 0, sizeof L);
    fill_ref_table(refs, n_refs, 0, &L.refs);
    L.n_refs = n_refs;
    L.width = width;
    L.q_ref = q_ref;
    L.res = res;
    L.n_q = n_q;
    L.cap = cap;
    L.out_offsets = out_offsets;
    L.out_pos = out_pos;
    L.capacity = out_pos ? out_pos_capacity : 0;
    L.partials = partials;
    return status_from_cuda(launch_locate(L, reinterpret_cast<cudaStream_t>(stream)));
}

int sa_save(const sa_index *idx, const char *path, void *stream) {
    if (!idx || !path) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t tb = (idx->nwords + SA_PAD_WORDS) * 8, sb = idx->n * (size_t)idx->width;
    const size_t kb = table_entries(idx->depth) * sizeof(uint4), lb = table_entries(idx->depth);
    std::vector<uint8_t> buf;
    try {
        buf.resize(tb + sb + kb + lb);
    } catch (...) {
        return SA_ERR_NOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(buf.data(), idx->text, tb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf.data() + tb, idx->sa, sb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf.data() + tb + sb, idx->keys, kb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf.data() + tb + sb + kb, idx->keylen, lb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from_cuda(e);
    FileHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.width = idx->width;
    h.n = idx->n;
    h.depth = idx->depth;
    h.kmer_k = idx->kmer_k;
    h.nwords = idx->nwords;
    h.checksum = fnv1a(14695981039346656037ull, buf.data(), buf.size());
    FILE *f = fopen(path, "wb");
    if (!f) return SA_ERR_IO;
    bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? SA_OK : SA_ERR_IO;
}

int sa_load(const char *path, void *stream, sa_index **out) {
    if (!path || !out) return SA_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    FILE *f = fopen(path, "rb");
    if (!f) return SA_ERR_IO;
    FileHeader h;
    if (fread(&h, sizeof h, 1, f) != 1) {
        fclose(f);
        return SA_ERR_FORMAT;
    }
    if (memcmp(h.magic, kMagic, 8) != 0 || h.version != 1 || (h.width != 4 && h.width != 8) || h.n == 0 ||
        h.n >= 0xFFFFFFFFull || h.nwords != (h.n + 31) / 32 || h.depth > SA_MAX_KEY_DEPTH || h.kmer_k > 15) {
        fclose(f);
        return SA_ERR_FORMAT;
    }
    sa_index *idx = new (std::nothrow) sa_index();
    if (!idx) {
        fclose(f);
        return SA_ERR_NOMEM;
    }
    cudaGetDevice(&idx->device);
    idx->n = h.n;
    idx->width = h.width;
    idx->depth = h.depth;
    idx->kmer_k = h.kmer_k;
    const size_t tb = (h.nwords + SA_PAD_WORDS) * 8, sb = h.n * (size_t)h.width;
    const size_t kb = table_entries(h.depth) * sizeof(uint4), lb = table_entries(h.depth);
    std::vector<uint8_t> buf;
    try {
        buf.resize(tb + sb + kb + lb);
    } catch (...) {
        fclose(f);
        delete idx;
        return SA_ERR_NOMEM;
    }
    const bool rd = fread(buf.data(), 1, buf.size(), f) == buf.size();
    fclose(f);
    if (!rd || fnv1a(14695981039346656037ull, buf.data(), buf.size()) != h.checksum) {
        delete idx;
        return SA_ERR_FORMAT;
    }
    int st = alloc_index(idx);
    if (st == SA_OK) st = alloc_search_arrays(idx);
    if (st) {
        free_index(idx);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(idx->text, buf.data(), tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx->sa, buf.data() + tb, sb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx->keys, buf.data() + tb + sb, kb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(idx->keylen, buf.data() + tb + sb + kb, lb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_build_records(idx, s);
    if (e == cudaSuccess) e = launch_build_kmer(idx, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaMemPoolTrimTo(scratch_pool(idx->device), 0);
    if (e != cudaSuccess) {
        free_index(idx);
        return status_from_cuda(e);
    }
    *out = idx;
    return SA_OK;
}

int sa_index_info(const sa_index *idx, uint64_t *n, uint32_t *width, uint32_t *key_depth, uint32_t *kmer_k,
                  uint64_t *device_bytes) {
    if (!idx) return SA_ERR_ARG;
    if (n) *n = idx->n;
    if (width) *width = idx->width;
    if (key_depth) *key_depth = idx->depth;
    if (kmer_k) *kmer_k = idx->kmer_k;
    if (device_bytes) *device_bytes = idx->device_bytes;
    return SA_OK;
}

int sa_copy_kmer_table(const sa_index *idx, void *dst, void *stream) {
    if (!idx || !dst || !idx->krt) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = ((1ull << (2 * idx->kmer_k)) + 1) * sizeof(uint32_t);
    if (on_device(dst)) return status_from_cuda(launch_copy_kmer_counts(idx, static_cast<uint32_t *>(dst), s));
    uint32_t *tmp = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void **>(&tmp), bytes, s);
    if (e != cudaSuccess) return status_from_cuda(e);
    e = launch_copy_kmer_counts(idx, tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, tmp, bytes, cudaMemcpyDeviceToHost, s);
    scratch_free(tmp, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return status_from_cuda(e);
}

int sa_copy_suffix_array(const sa_index *idx, void *dst, void *stream) {
    if (!idx || !dst) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dst, idx->sa, idx->n * (size_t)idx->width, cudaMemcpyDefault, s);
    return status_from_cuda(e);
}

void sa_free(sa_index *idx) {
    if (!idx) return;
    cudaDeviceSynchronize();
    free_index(idx);
}

int sa_suffix_array_gpu(const char *text, uint64_t n, uint32_t width, uint32_t flags, void *sa_out, void *stream) {
    NvtxRange range("sa_suffix_array_gpu");
    if (!text || !sa_out || n == 0 || n >= 0xFFFFFFFFull || (width != 4 && width != 8) || (flags & ~SA_BUILD_DC3))
        return SA_ERR_ARG;
    if (!on_device(sa_out)) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    sa_index tmp;  // a text and a suffix array only: what the builders read and write
    memset(&tmp, 0, sizeof tmp);
    tmp.n = n;
    tmp.width = width;
    tmp.nwords = (n + 31) / 32;
    tmp.sa = sa_out;
    if (cudaGetDevice(&tmp.device) != cudaSuccess) return SA_ERR_CUDA;
    int st = SA_OK;
    {
        Scratch sc{s};
        cudaError_t err = cudaSuccess;
        const char *text_d = device_view(text, n, sc, &err);
        tmp.text = sc.get<uint64_t>(tmp.nwords + SA_PAD_WORDS);
        int *flag = sc.get<int>(1);
        if (sc.failed) return SA_ERR_NOMEM;
        int hflag = 0;
        if (err == cudaSuccess) err = cudaMemsetAsync(flag, 0, sizeof(int), s);
        if (err == cudaSuccess) err = launch_pack_text(text_d, n, tmp.text, tmp.nwords + SA_PAD_WORDS, flag, s);
        if (err == cudaSuccess) err = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return status_from_cuda(err);
        if (hflag) return SA_ERR_BASE;
        st = (flags & SA_BUILD_DC3) ? build_suffix_array_dc3(&tmp, s) : build_suffix_array(&tmp, s);
        cudaStreamSynchronize(s);
    }
    cudaMemPoolTrimTo(scratch_pool(tmp.device), 0);
    return st;
}

int sa_search_order(const sa_index *const *refs, uint32_t n_refs, uint64_t n_q, const sa_search_params *params,
                    int *kmer_order) {
    uint32_t width = 0;
    int st = check_refs(refs, n_refs, &width);
    if (st) return st;
    if (!kmer_order) return SA_ERR_ARG;
    const uint32_t order = params ? params->flags & (SA_PARAM_KMER_ORDER | SA_PARAM_INPUT_ORDER) : 0u;
    if (order == (SA_PARAM_KMER_ORDER | SA_PARAM_INPUT_ORDER)) return SA_ERR_ARG;
    *kmer_order = use_kmer_order(refs, n_refs, n_q, order) ? 1 : 0;
    return SA_OK;
}

int sa_scratch_info(uint64_t *reserved_bytes, uint64_t *used_bytes, uint64_t *used_high_bytes, int reset_high) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SA_ERR_CUDA;
    cudaMemPool_t pool = scratch_pool(dev);
    if (!pool) return SA_ERR_CUDA;
    uint64_t v = 0;  // the attributes are 64-bit (cuuint64_t)
    if (reserved_bytes) {
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess) return SA_ERR_CUDA;
        *reserved_bytes = v;
    }
    if (used_bytes) {
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) != cudaSuccess) return SA_ERR_CUDA;
        *used_bytes = v;
    }
    if (used_high_bytes) {
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v) != cudaSuccess) return SA_ERR_CUDA;
        *used_high_bytes = v;
    }
    if (reset_high) {
        uint64_t zero = 0;
        if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero) != cudaSuccess) return SA_ERR_CUDA;
    }
    return SA_OK;
}

const char *sa_strerror(int status) {
    switch (status) {
        case SA_OK: return "success";
        case SA_ERR_ARG: return "invalid argument";
        case SA_ERR_BASE: return "byte outside {A,C,G,T,a,c,g,t}";
        case SA_ERR_NOMEM: return "out of memory";
        case SA_ERR_CUDA: return "CUDA runtime error";
        case SA_ERR_TIMEOUT: return "bounded device wait timed out";
        case SA_ERR_CAPACITY: return "output buffer too small";
        case SA_ERR_IO: return "file I/O error";
        case SA_ERR_FORMAT: return "not an index file or checksum mismatch";
        default: return "unknown status";
    }
}

uint32_t sa_version(void) { return 0x000100u; }

}  // extern "C"
