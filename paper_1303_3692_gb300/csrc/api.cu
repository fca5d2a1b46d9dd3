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
    for (uint32_t r = 0; r < n_refs; r++) {
        const sa_index *x = refs[r];
        RefDesc &d = t->r[r];
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

int search_impl(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                const uint32_t *q_ref, uint64_t n_q, sa_result *out, void *stream, const sa_search_params *params,
                bool plain) {
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
    const bool out_dev = on_device(out);
    sa_result *out_d = out_dev ? out : sc.get<sa_result>(n_q);
    const uint64_t nwords = (total + 31) / 32;
    uint64_t *tq = sc.get<uint64_t>(nwords + SA_TQ_PAD_WORDS);
    uint32_t *tv = sc.get<uint32_t>(nwords + SA_TQ_PAD_WORDS);
    uint4 *wrec = plain ? nullptr : sc.get<uint4>(4 * n_q);
    int *flags = sc.get<int>(4);  // [0] pack error, [1] status, [2] worklist count, [3] bad reference id
    unsigned long long *counter = sc.get<unsigned long long>(1);
    if (sc.failed) return SA_ERR_NOMEM;
    if (err != cudaSuccess) return status_from_cuda(err);
    if (((uintptr_t)wrec & 31u) != 0) return SA_ERR_CUDA;  // the search reads 32-byte records
    if ((err = cudaMemsetAsync(flags, 0, 4 * sizeof(int), s)) != cudaSuccess) return status_from_cuda(err);
    if ((err = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return status_from_cuda(err);

    SearchLaunch L;
    memset(&L, 0, sizeof L);
    const uint32_t threads = params && params->threads_per_block ? params->threads_per_block : 1024;
    const uint32_t bps = params && params->blocks_per_sm ? params->blocks_per_sm : 1;
    if (threads < 32 || threads > 1024 || threads % 32 || bps == 0 || threads * bps > 2048) return SA_ERR_ARG;
    // shared memory per SM is 228 KB; each CTA also holds ~4 KB of descriptors
    const uint32_t per_cta = 224u * 1024u / bps - 6144u;
    const uint32_t budget = per_cta < kSmemBudget ? per_cta : kSmemBudget;
    const uint32_t want_depth = params && params->key_depth ? params->key_depth : kDefaultDepth;
    L.smem_bytes = fill_ref_table(refs, n_refs, plain ? 0 : want_depth, &L.refs, budget);
    L.n_refs = n_refs;
    L.width = width;
    L.ascii = bases_d;
    L.tq = tq;
    L.tv = tv;
    L.nwords = nwords;
    L.q_off = off_d;
    L.first = first;
    L.total = total;
    L.q_ref = ref_d;
    L.n_q = n_q;
    L.wrec = wrec;
    L.wl_count = reinterpret_cast<uint32_t *>(flags + 2);
    L.out = out_d;
    L.pack_err = flags;
    L.counter = counter;
    L.status = flags + 1;
    const int sms = device_sm_count();
    L.threads = threads;
    L.blocks = (uint32_t)sms * bps;
    L.chunk = params && params->chunk ? params->chunk : 64;
    L.front_probes = params && params->front_probes ? params->front_probes : default_front_probes(refs, n_refs);
    L.revcomp = params && (params->flags & SA_PARAM_REVERSE_COMPLEMENT);
    L.expire_waits = params && (params->flags & SA_PARAM_EXPIRE_WAITS);
    L.bad_ref = flags + 3;
    if (L.front_probes > 64) return SA_ERR_ARG;
    int *dstatus = params ? params->device_status : nullptr;
    if (dstatus && !on_device(dstatus)) return SA_ERR_ARG;

    if ((err = launch_pack_batch(L, tq, tv, s)) != cudaSuccess) return status_from_cuda(err);
    cudaEvent_t ev0 = params ? reinterpret_cast<cudaEvent_t>(params->search_events[0]) : nullptr;
    cudaEvent_t ev1 = params ? reinterpret_cast<cudaEvent_t>(params->search_events[1]) : nullptr;
    if (ev0 && (err = cudaEventRecord(ev0, s)) != cudaSuccess) return status_from_cuda(err);
    if (plain) {
        err = launch_search_plain(L, s);
    } else {
        err = launch_front(L, s);
        if (err == cudaSuccess) err = launch_search(L, s);
    }
    if (err != cudaSuccess) return status_from_cuda(err);
    if (ev1 && (err = cudaEventRecord(ev1, s)) != cudaSuccess) return status_from_cuda(err);
    if (dstatus && (err = launch_search_status(flags, dstatus, s)) != cudaSuccess) return status_from_cuda(err);
    if (!out_dev) {
        int hflags[4] = {0, 0, 0, 0};
        if ((err = cudaMemcpyAsync(out, out_d, n_q * sizeof(sa_result), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        if ((err = cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return status_from_cuda(err);
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return status_from_cuda(err);
        if (hflags[1]) return hflags[1];
        if (hflags[0]) return SA_ERR_BASE;
        if (hflags[3]) return SA_ERR_ARG;
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

using namespace sa;

extern "C" {

int sa_build(const char *text, uint64_t n, uint32_t flags, void *stream, sa_index **out) {
    NvtxRange range("sa_build");
    if (!out) return SA_ERR_ARG;
    *out = nullptr;
    if (!text || n == 0 || n >= 0xFFFFFFFFull) return SA_ERR_ARG;
    const uint32_t wflags = flags & (SA_W32 | SA_W64);
    if (wflags != SA_W32 && wflags != SA_W64) return SA_ERR_ARG;
    if (flags & ~(SA_W32 | SA_W64 | SA_NO_KMER | SA_BUILD_HOST | SA_KMER_K(15))) return SA_ERR_ARG;
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

int sa_search_batch(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                    const uint32_t *q_ref, uint64_t n_q, sa_result *out, void *stream) {
    return search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, nullptr, false);
}

int sa_search_batch_ex(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                       const uint32_t *q_ref, uint64_t n_q, sa_result *out, void *stream,
                       const sa_search_params *params) {
    return search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, params, false);
}

int sa_search_batch_plain(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                          const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q, sa_result *out,
                          void *stream) {
    return search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, nullptr, true);
}

namespace sa {

int locate_impl(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref, const sa_result *res,
                uint64_t n_q, uint32_t cap, uint64_t *out_offsets, void *out_pos, uint64_t out_pos_capacity,
                void *stream, int *dstatus = nullptr) {
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
    const uint64_t tiles = locate_tiles(n_q);
    uint64_t *partials = sc.get<uint64_t>(tiles + 1);
    int *overflow = dstatus && pos_d ? sc.get<int>(1) : nullptr;
    if (sc.failed) return SA_ERR_NOMEM;
    if (err != cudaSuccess) return status_from_cuda(err);
    if (overflow && (err = cudaMemsetAsync(overflow, 0, sizeof(int), s)) != cudaSuccess) return status_from_cuda(err);
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
    L.capacity = pos_d ? out_pos_capacity : 0;
    L.partials = partials;
    L.overflow = overflow;
    if ((err = launch_locate(L, s)) != cudaSuccess) return status_from_cuda(err);
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

}  // namespace sa

int sa_locate(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref, const sa_result *res,
              uint64_t n_q, uint32_t cap, uint64_t *out_offsets, void *out_pos, uint64_t out_pos_capacity,
              void *stream) {
    return sa::locate_impl(refs, n_refs, q_ref, res, n_q, cap, out_offsets, out_pos, out_pos_capacity, stream);
}

int sa_search_locate(const sa_index *const *refs, uint32_t n_refs, const char *q_bases, const uint64_t *q_offsets,
                     const uint32_t *q_ref, uint64_t n_q, sa_result *out, uint32_t cap, uint64_t *out_offsets,
                     void *out_pos, uint64_t out_pos_capacity, void *stream, const sa_search_params *params) {
    using namespace sa;
    NvtxRange range("sa_search_locate");
    if (!out_offsets || (n_q && !out)) return SA_ERR_ARG;
    const int st = search_impl(refs, n_refs, q_bases, q_offsets, q_ref, n_q, out, stream, params, false);
    if (st && st != SA_ERR_BASE && st != SA_ERR_ARG) return st;
    // invalid queries carry the all-ones result (no positions); the rest are located
    int *dstatus = params ? params->device_status : nullptr;
    const int lst =
        locate_impl(refs, n_refs, q_ref, out, n_q, cap, out_offsets, out_pos, out_pos_capacity, stream, dstatus);
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
