// locate.cu -- text positions of the matches: out_offsets is the exclusive
// prefix sum of k_q = min(count_q, cap) and query q's first k_q suffix-array
// entries SA[lo_q], SA[lo_q + 1], ... are copied to out_pos[out_offsets[q]..].
// (The paper reports only [LB, RB]; locate is an extension of it.)
//
// Three launches: per-tile sums of k_q, one CTA scanning the tile sums, and a
// CTA per tile that scans its own k_q, writes the offsets and gathers.  Each
// tile is kTileThreads x kItems consecutive queries; thread t of a tile owns
// queries t, t + kTileThreads, t + 2 kTileThreads, ... of it.
#include <mutex>

#include "sa_internal.cuh"

// Scratch of sa_locate_noalloc: one partial sum per 4096-query tile of the
// largest accepted batch, plus the total (131,080 bytes).  Every device that
// loads the library holds it until exit.  Host code must pass its device
// address (from cudaGetSymbolAddress), never the symbol itself.
static __device__ __align__(256) uint64_t g_noalloc_partials[SA_LOCATE_NOALLOC_MAX_QUERIES / 4096 + 1];

namespace sa {

namespace {

constexpr int kTileThreads = 512;
constexpr int kItems = 8;
constexpr uint64_t kTile = (uint64_t)kTileThreads * kItems;

__device__ __forceinline__ uint64_t kept(const sa_result &r, uint32_t cap) {
    if (r.count == ~0ull) return 0;  // invalid query (reported as all-ones)
    return r.count < cap ? r.count : cap;
}

// Exclusive block scan of one value per thread; returns the block total in *total.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total) {
    __shared__ uint64_t warp_sums[32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const unsigned nw = blockDim.x >> 5;
        uint64_t w = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (unsigned)o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    const uint64_t before = warp ? warp_sums[warp - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kTileThreads) tile_sums_kernel(const sa_result *__restrict__ res, uint64_t n_q,
                                                                  uint32_t cap, uint64_t *partials) {
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const uint64_t q = base + threadIdx.x + (uint64_t)i * kTileThreads;
        if (q < n_q) s += kept(res[q], cap);
    }
    uint64_t total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// One CTA: exclusive scan of the tile sums in place; partials[ntiles] = total.
__global__ void __launch_bounds__(1024) scan_partials_kernel(uint64_t *partials, uint64_t ntiles) {
    __shared__ uint64_t carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (uint64_t base = 0; base < ntiles; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t v = i < ntiles ? partials[i] : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, &total);
        const uint64_t carry = carry_s;
        if (i < ntiles) partials[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + total;
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[ntiles] = carry_s;
}

// Item i of thread t covers query tile_base + i * kTileThreads + t (the same
// queries tile_sums_kernel summed), so every load of results and every store
// of offsets is coalesced.  Items are scanned in order i = 0..kItems-1.
template <typename IdxT>
__global__ void __launch_bounds__(kTileThreads) tile_gather_kernel(const __grid_constant__ LocateLaunch a) {
    const uint64_t tile_base = (uint64_t)blockIdx.x * kTile;
    const uint64_t ntiles = gridDim.x;
    if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) a.out_offsets[a.n_q] = a.partials[ntiles];
    uint64_t running = a.partials[blockIdx.x];
    IdxT *pos = reinterpret_cast<IdxT *>(a.out_pos);
#pragma unroll 1
    for (int i = 0; i < kItems; i++) {
        const uint64_t q = tile_base + (uint64_t)i * kTileThreads + threadIdx.x;
        sa_result r{0, 0, 0};
        if (q < a.n_q) r = a.res[q];
        const uint64_t k = q < a.n_q ? kept(r, a.cap) : 0;
        uint64_t total;
        const uint64_t off = running + block_exclusive_scan(k, &total);
        running += total;
        if (q >= a.n_q) continue;
        a.out_offsets[q] = off;
        if (pos != nullptr && k != 0) {
            const uint32_t ref = a.q_ref ? a.q_ref[q] : 0u;
            const RefDesc &d = a.refs.r[ref < a.n_refs ? ref : 0];
            const IdxT *sa = reinterpret_cast<const IdxT *>(d.sa);
            const uint64_t kk = (ref < a.n_refs && r.lo <= d.n && k <= d.n - r.lo) ? k : 0;  // never read past SA
            for (uint64_t t = 0; t < kk; t++) {
                if (off + t < a.capacity) pos[off + t] = __ldg(sa + r.lo + t);
            }
        }
    }
}

}  // namespace

uint64_t locate_tiles(uint64_t n_q) { return (n_q + kTile - 1) / kTile; }

static_assert(kTile == 4096, "the static scratch below is sized for 4096-query tiles");

cudaError_t locate_static_partials(uint64_t **ptr, uint64_t *entries) {
    static std::mutex mu;
    static uint64_t *addr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        addr[dev] = reinterpret_cast<uint64_t *>(p);
    }
    *ptr = addr[dev];
    *entries = SA_LOCATE_NOALLOC_MAX_QUERIES / 4096 + 1;
    return cudaSuccess;
}


cudaError_t launch_locate(const LocateLaunch &L, cudaStream_t s) {
    const uint64_t tiles = locate_tiles(L.n_q);
    if (tiles == 0) {
        return cudaMemsetAsync(L.out_offsets, 0, sizeof(uint64_t), s);
    }
    tile_sums_kernel<<<(unsigned)tiles, kTileThreads, 0, s>>>(L.res, L.n_q, L.cap, L.partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(L.partials, tiles);
    if (L.width == 4)
        tile_gather_kernel<uint32_t><<<(unsigned)tiles, kTileThreads, 0, s>>>(L);
    else
        tile_gather_kernel<uint64_t><<<(unsigned)tiles, kTileThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace sa
