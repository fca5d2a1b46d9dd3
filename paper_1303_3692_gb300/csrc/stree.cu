// stree.cu -- a flattened suffix tree of an index's text and its search on
// the GPU: the paper's comparison index (Section III defines the suffix tree;
// Table V times a GPU suffix-tree search beside the suffix-array one).  It
// answers the same question -- the suffix-array interval [lo, hi) of every
// query, misses at their insertion point -- so its results equal the suffix
// array search's exactly.
//
// The tree's internal nodes are the LCP intervals of the suffix array: an
// interval [lb, rb] of ranks whose suffixes share l = min LCP(lb+1..rb) bases
// and split at base l.  Leaves are single ranks.  Built here:
//   1. the LCP array on the GPU (lcp_kernel: each adjacent pair of suffixes
//      compared 32 bases at a time on the packed text);
//   2. the tree on the host from SA and LCP by the bottom-up traversal of LCP
//      intervals (a stack; each interval is closed when the LCP drops below
//      its depth, and becomes the parent of the intervals closed inside it);
//   3. the nodes flattened into one array of 32-byte records {lb, rb, depth,
//      pos, child[A], child[C], child[G], child[T]} (pos = SA[lb], a text
//      position of the node's path label; a child is a node index, a leaf
//      rank with the top bit set, or none), uploaded.
// The search (stree_search_kernel) runs one thread per query from the root:
// at a node of string depth d it follows the child of the query's base d and
// compares the query with that edge's bases in the text, 32 at a time, until
// the query ends (its interval is the child's), the edge ends (descend), or a
// base differs (a miss: the insertion point is the child's first rank when
// the query is smaller, one past its last when larger).  Each step is a
// dependent node read and a text read: the work the paper's Table V
// contrasts with the suffix array's binary search.
#include <algorithm>
#include <new>
#include <vector>

#include "sa_internal.cuh"

struct sa_stree {
    uint64_t n;
    uint64_t n_nodes;
    uint32_t root;
    int device;
    const sa_index *idx;  // the text and suffix array the tree indexes
    uint4 *nodes;         // device: n_nodes records of 32 bytes (2 uint4)
    uint64_t device_bytes;
};

namespace sa {

namespace {

constexpr uint32_t kLeaf = 0x80000000u;
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kThreads = 256;

// LCP[i] = length of the common prefix of the suffixes at ranks i - 1 and i
// (LCP[0] = 0).
template <typename IdxT>
__global__ void lcp_kernel(const uint64_t *__restrict__ T, uint64_t n, const IdxT *__restrict__ sa, uint32_t *lcp) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (i == 0) {
            lcp[0] = 0;
            continue;
        }
        const uint64_t a = sa[i - 1], b = sa[i];
        const uint64_t room = n - (a > b ? a : b);  // bases both suffixes have
        uint64_t l = 0;
        while (l < room) {
            const uint64_t x = text_window(T, a + l) ^ text_window(T, b + l);
            const uint64_t d = x ? (uint64_t)(__clzll((long long)x) >> 1) : 32u;
            if (d < 32) {
                l += d;
                break;
            }
            l += 32;
        }
        lcp[i] = (uint32_t)(l < room ? l : room);
    }
}

// The query (bases qa.. of the packed batch, m of them) against the bases of
// the text from position p, from offset `from` up to offset `to` (to <= m and
// p + to <= n): the first offset where they differ, or `to`; *less is set when
// the query's base there is the smaller.
__device__ __forceinline__ uint32_t edge_match(const uint64_t *__restrict__ T, uint64_t p,
                                               const uint64_t *__restrict__ tq, uint64_t qa, uint32_t from,
                                               uint32_t to, bool *less) {
    uint32_t off = from;
    while (off < to) {
        const uint64_t q = text_window(tq, qa + off), t = text_window(T, p + off);
        const uint64_t x = q ^ t;
        const uint32_t d = x ? ((uint32_t)__clzll((long long)x) >> 1) : 32u;
        const uint32_t span = to - off < 32u ? to - off : 32u;
        if (d < span) {
            *less = q < t;
            return off + d;
        }
        off += span;
    }
    return to;
}

template <typename IdxT>
__global__ void stree_search_kernel(const uint4 *__restrict__ nodes, uint32_t root, const uint64_t *__restrict__ T,
                                    const IdxT *__restrict__ sa, uint64_t n, const uint64_t *__restrict__ q_off,
                                    uint64_t first, uint64_t total, const uint64_t *__restrict__ tq,
                                    const uint32_t *__restrict__ tv, uint64_t n_q, sa_result *out, int *bad_flag) {
    const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_q) return;
    const uint64_t a0 = __ldg(q_off + q) - first, a1 = __ldg(q_off + q + 1) - first;
    bool bad = !(a0 <= a1 && a1 <= total && a1 - a0 < (1ull << 31));
    if (!bad)
        for (uint64_t b = a0; b < a1; b++)
            if ((__ldg(tv + (b >> 5)) >> (b & 31u)) & 1u) bad = true;
    if (bad) {
        atomicOr(bad_flag, 1);
        store_result(out, q, ~0ull, ~0ull, ~0u);
        return;
    }
    const uint32_t m = (uint32_t)(a1 - a0);
    uint4 lo_half = __ldg(nodes + 2 * (size_t)root), hi_half = __ldg(nodes + 2 * (size_t)root + 1);
    uint32_t depth = lo_half.z;  // bases matched: the current node's string depth
    for (;;) {
        if (depth >= m) {  // the query ends at this node
            store_result(out, q, lo_half.x, (uint64_t)lo_half.y + 1, ~0u);
            return;
        }
        const uint64_t c = (__ldg(tq + ((a0 + depth) >> 5)) >> (62u - 2u * (uint32_t)((a0 + depth) & 31u))) & 3u;
        const uint32_t ch = c == 0 ? hi_half.x : c == 1 ? hi_half.y : c == 2 ? hi_half.z : hi_half.w;
        if (ch == kNone) {  // no suffix continues with this base: insert before the first larger child
            uint64_t ip = (uint64_t)lo_half.y + 1;
            for (uint32_t cc = (uint32_t)c + 1; cc < 4; cc++) {
                const uint32_t x = cc == 1 ? hi_half.y : cc == 2 ? hi_half.z : hi_half.w;
                if (x == kNone) continue;
                ip = (x & kLeaf) ? (x & ~kLeaf) : __ldg(nodes + 2 * (size_t)x).x;
                break;
            }
            store_result(out, q, ip, ip, ~0u);
            return;
        }
        uint32_t clb, crb, cdepth;
        uint64_t cpos;
        uint4 nlo = make_uint4(0, 0, 0, 0), nhi = make_uint4(0, 0, 0, 0);
        if (ch & kLeaf) {
            clb = crb = ch & ~kLeaf;
            cpos = sa[clb];
            cdepth = (uint32_t)(n - cpos);
        } else {
            nlo = __ldg(nodes + 2 * (size_t)ch);
            nhi = __ldg(nodes + 2 * (size_t)ch + 1);
            clb = nlo.x;
            crb = nlo.y;
            cdepth = nlo.z;
            cpos = nlo.w;
        }
        const uint32_t to = cdepth < m ? cdepth : m;
        bool less = false;
        const uint32_t l = edge_match(T, cpos, tq, a0, depth, to, &less);
        if (l < to) {  // a base differs on the edge
            const uint64_t ip = less ? clb : (uint64_t)crb + 1;
            store_result(out, q, ip, ip, ~0u);
            return;
        }
        if (m <= cdepth) {  // the query ends on this edge
            store_result(out, q, clb, (uint64_t)crb + 1, ~0u);
            return;
        }
        if (ch & kLeaf) {  // the suffix ends before the query: it sorts first
            store_result(out, q, (uint64_t)crb + 1, (uint64_t)crb + 1, ~0u);
            return;
        }
        lo_half = nlo;
        hi_half = nhi;
        depth = cdepth;
    }
}

struct HostNode {
    uint32_t lb, rb, depth, pos;
    uint32_t child[4];
};

// Base code of text position p of the packed text (p < n).
inline uint32_t base_at(const std::vector<uint64_t> &T, uint64_t p) { return (uint32_t)(T[p >> 5] >> (62 - 2 * (p & 31))) & 3u; }

// The LCP-interval tree of (SA, LCP), flattened; returns the root's index.
uint32_t build_nodes(const std::vector<uint64_t> &T, uint64_t n, const std::vector<uint64_t> &sa,
                     const std::vector<uint32_t> &lcp, std::vector<HostNode> &nodes) {
    struct Frame {
        uint32_t lcp, lb;
        std::vector<uint32_t> kids;  // node indices of the child intervals closed so far, in rank order
    };
    std::vector<Frame> st;
    st.push_back(Frame{0, 0, {}});
    auto close = [&](Frame &f, uint32_t rb) -> uint32_t {
        HostNode h;
        h.lb = f.lb;
        h.rb = rb;
        h.depth = f.lcp;
        h.pos = (uint32_t)sa[f.lb];
        for (auto &c : h.child) c = kNone;
        // children: the closed child intervals, and single ranks (leaves) between them
        size_t k = 0;
        for (uint64_t r = f.lb; r <= rb;) {
            uint32_t id, first;
            if (k < f.kids.size() && nodes[f.kids[k]].lb == r) {
                id = f.kids[k];
                first = (uint32_t)r;
                r = (uint64_t)nodes[f.kids[k]].rb + 1;
                k++;
            } else {
                id = kLeaf | (uint32_t)r;
                first = (uint32_t)r;
                r++;
            }
            const uint64_t p = sa[first] + f.lcp;
            if (p < n) h.child[base_at(T, p)] = id;  // a suffix of exactly depth bases has no next base
        }
        nodes.push_back(h);
        return (uint32_t)(nodes.size() - 1);
    };
    uint32_t last = kNone;
    for (uint64_t i = 1; i <= n; i++) {
        const int64_t cur = i < n ? (int64_t)lcp[i] : -1;
        uint32_t lb = (uint32_t)(i - 1);
        last = kNone;
        while (!st.empty() && cur < (int64_t)st.back().lcp) {
            Frame f = std::move(st.back());
            st.pop_back();
            last = close(f, (uint32_t)(i - 1));
            lb = nodes[last].lb;
            if (!st.empty() && cur <= (int64_t)st.back().lcp) {
                st.back().kids.push_back(last);
                last = kNone;
            }
        }
        if (!st.empty() && cur > (int64_t)st.back().lcp) {
            Frame f{(uint32_t)cur, lb, {}};
            if (last != kNone) f.kids.push_back(last);
            st.push_back(std::move(f));
        } else if (st.empty()) {
            break;  // the root closed: i == n
        }
    }
    return last;  // the root is closed last
}

}  // namespace

}  // namespace sa

using namespace sa;

extern "C" {

int sa_stree_build(const sa_index *idx, void *stream, sa_stree **out) {
    if (!idx || !out) return SA_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t n = idx->n;
    if (n >= (uint64_t)kLeaf) return SA_ERR_ARG;  // a child names a rank with the top bit clear
    std::vector<uint64_t> T, sa_h;
    std::vector<uint32_t> lcp_h;
    std::vector<HostNode> nodes;
    try {
        T.resize(idx->nwords + SA_PAD_WORDS);
        sa_h.resize(n);
        lcp_h.resize(n);
        nodes.reserve(n);
    } catch (const std::bad_alloc &) {
        return SA_ERR_NOMEM;
    }
    uint32_t *lcp_d = nullptr;
    cudaError_t e = scratch_alloc(reinterpret_cast<void **>(&lcp_d), n * sizeof(uint32_t), s);
    if (e != cudaSuccess) return status_from_cuda(e);
    uint64_t blocks = (n + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)device_sm_count() * 32;
    if (blocks > cap) blocks = cap;
    if (idx->width == 4)
        lcp_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(idx->text, n, reinterpret_cast<const uint32_t *>(idx->sa), lcp_d);
    else
        lcp_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(idx->text, n, reinterpret_cast<const uint64_t *>(idx->sa), lcp_d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(lcp_h.data(), lcp_d, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(T.data(), idx->text, T.size() * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && idx->width == 8)
        e = cudaMemcpyAsync(sa_h.data(), idx->sa, n * 8, cudaMemcpyDeviceToHost, s);
    std::vector<uint32_t> sa32;
    if (e == cudaSuccess && idx->width == 4) {
        try {
            sa32.resize(n);
        } catch (const std::bad_alloc &) {
            scratch_free(lcp_d, s);
            return SA_ERR_NOMEM;
        }
        e = cudaMemcpyAsync(sa32.data(), idx->sa, n * 4, cudaMemcpyDeviceToHost, s);
    }
    scratch_free(lcp_d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (idx->width == 4)
        for (uint64_t i = 0; i < n; i++) sa_h[i] = sa32[i];
    uint32_t root = 0;
    try {
        root = build_nodes(T, n, sa_h, lcp_h, nodes);
    } catch (const std::bad_alloc &) {
        return SA_ERR_NOMEM;
    }
    sa_stree *t = new (std::nothrow) sa_stree();
    if (!t) return SA_ERR_NOMEM;
    t->n = n;
    t->n_nodes = nodes.size();
    t->root = root;
    t->idx = idx;
    cudaGetDevice(&t->device);
    t->device_bytes = nodes.size() * sizeof(HostNode);
    static_assert(sizeof(HostNode) == 32, "a node is two uint4");
    if (cudaMalloc(&t->nodes, t->device_bytes) != cudaSuccess) {
        cudaGetLastError();
        delete t;
        return SA_ERR_NOMEM;
    }
    e = cudaMemcpyAsync(t->nodes, nodes.data(), t->device_bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(t->nodes);
        delete t;
        return status_from_cuda(e);
    }
    *out = t;
    return SA_OK;
}

int sa_stree_search(const sa_stree *t, const char *q_bases, const uint64_t *q_offsets, uint64_t n_q, sa_result *out,
                    void *stream) {
    if (!t || !q_offsets || !out || n_q >= (1ull << 32)) return SA_ERR_ARG;
    if (n_q == 0) return SA_OK;
    cudaPointerAttributes at;
    auto dev = [&](const void *p) {
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    };
    // device inputs and outputs only: the comparison index is a measurement tool
    if (!dev(q_offsets) || !dev(out) || (q_bases && !dev(q_bases)) || ((uintptr_t)out & 31u)) return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint64_t fl[2];
    cudaError_t e = cudaMemcpyAsync(&fl[0], q_offsets, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fl[1], q_offsets + n_q, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (fl[1] < fl[0] || (fl[1] > fl[0] && !q_bases)) return SA_ERR_ARG;
    const uint64_t total = fl[1] - fl[0], nwords = (total + 31) / 32;
    uint64_t *tq = nullptr;
    uint32_t *tv = nullptr;
    int *flag = nullptr;
    e = scratch_alloc(reinterpret_cast<void **>(&tq), (nwords + SA_TQ_PAD_WORDS) * 8, s);
    if (e == cudaSuccess) e = scratch_alloc(reinterpret_cast<void **>(&tv), (nwords + SA_TQ_PAD_WORDS) * 4, s);
    if (e == cudaSuccess) e = scratch_alloc(reinterpret_cast<void **>(&flag), sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        SearchLaunch L;
        memset(&L, 0, sizeof L);
        L.ascii = q_bases ? q_bases + fl[0] : nullptr;
        L.total = total;
        L.nwords = nwords;
        e = launch_pack_batch(L, tq, tv, s);
    }
    if (e == cudaSuccess) {
        const unsigned blocks = (unsigned)((n_q + kThreads - 1) / kThreads);
        if (t->idx->width == 4)
            stree_search_kernel<<<blocks, kThreads, 0, s>>>(t->nodes, t->root, t->idx->text,
                                                            reinterpret_cast<const uint32_t *>(t->idx->sa), t->n,
                                                            q_offsets, fl[0], total, tq, tv, n_q, out, flag);
        else
            stree_search_kernel<<<blocks, kThreads, 0, s>>>(t->nodes, t->root, t->idx->text,
                                                            reinterpret_cast<const uint64_t *>(t->idx->sa), t->n,
                                                            q_offsets, fl[0], total, tq, tv, n_q, out, flag);
        e = cudaGetLastError();
    }
    scratch_free(tq, s);
    scratch_free(tv, s);
    scratch_free(flag, s);
    return status_from_cuda(e);
}

int sa_stree_info(const sa_stree *t, uint64_t *nodes, uint64_t *device_bytes) {
    if (!t) return SA_ERR_ARG;
    if (nodes) *nodes = t->n_nodes;
    if (device_bytes) *device_bytes = t->device_bytes;
    return SA_OK;
}

void sa_stree_free(sa_stree *t) {
    if (!t) return;
    cudaDeviceSynchronize();
    cudaFree(t->nodes);
    delete t;
}

}  // extern "C"
