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

// One CTA: exclusive scan of the tile sums in place, starting from *base_in
// (0 when null); partials[ntiles] = base + total.
__global__ void __launch_bounds__(1024) scan_partials_kernel(uint64_t *partials, uint64_t ntiles,
                                                             const uint64_t *base_in) {
    __shared__ uint64_t carry_s;
    if (threadIdx.x == 0) carry_s = base_in ? *base_in : 0;
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

// One CTA per tile of kTile queries; warp w owns the tile's queries
// [w * 256, w * 256 + 256), lane l its queries w * 256 + i * 32 + l for
// i < kItems, so every load of results and store of offsets is coalesced.  A
// first pass reads the lane's results once and sums its items, keeping each
// item's count and lower bound in shared memory; one exchange of warp totals
// (one barrier) places the warps within the tile; a second pass places each
// item within the warp's run by a warp scan (shuffles), writes its offset and
// copies its positions.
template <typename IdxT>
__global__ void __launch_bounds__(kTileThreads, 3) tile_gather_kernel(const __grid_constant__ LocateLaunch a) {
    constexpr int kWarps = kTileThreads / 32;
    __shared__ uint64_t s_warp[kWarps];
    // each item's kept count and lower bound from the first pass (32 KB), so
    // the second pass does not read the results again: at 3.1 Gbp the L2 no
    // longer holds them by then
    __shared__ uint32_t s_k[kItems][kTileThreads];
    __shared__ uint32_t s_lo[kItems][kTileThreads];
    const uint64_t tile_base = (uint64_t)blockIdx.x * kTile;
    const uint64_t ntiles = gridDim.x;
    if (blockIdx.x == ntiles - 1 && threadIdx.x == 0) a.out_offsets[a.n_q] = a.partials[ntiles];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint64_t warp_base = tile_base + (uint64_t)warp * (32 * kItems);
    IdxT *pos = reinterpret_cast<IdxT *>(a.out_pos);

    uint64_t lane_sum = 0;
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const uint64_t q = warp_base + (uint64_t)i * 32 + lane;
        uint32_t k = 0, lo = 0xFFFFFFFFu;  // ranks are below 2^32 - 1: 0xFFFFFFFF copies nothing
        if (q < a.n_q) {
            const sa_result r = a.res[q];
            k = (uint32_t)kept(r, a.cap);  // cap is 32-bit
            if (r.lo < 0xFFFFFFFFull) lo = (uint32_t)r.lo;
        }
        s_k[i][threadIdx.x] = k;
        s_lo[i][threadIdx.x] = lo;
        lane_sum += k;
    }
    uint64_t tot = lane_sum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    if (lane == 0) s_warp[warp] = tot;
    __syncthreads();
    uint64_t run = a.partials[blockIdx.x];
    for (unsigned w = 0; w < warp; w++) run += s_warp[w];

    // Second pass over the items, from shared memory.
#pragma unroll
    for (int i = 0; i < kItems; i++) {
        const uint64_t q = warp_base + (uint64_t)i * 32 + lane;
        const uint32_t k = s_k[i][threadIdx.x];
        const uint64_t lo = s_lo[i][threadIdx.x];
        uint64_t x = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        const uint64_t off = run + x - k;
        run += __shfl_sync(0xFFFFFFFFu, x, 31);
        if (q >= a.n_q) continue;
        a.out_offsets[q] = off;
        if (pos == nullptr || k == 0) continue;
        const uint32_t ref = a.q_ref ? (a.q_ref[q] & ~kStrandBit) : 0u;  // bit 31: the strand, not the reference
        const RefDesc &d = a.refs.r[ref < a.n_refs ? ref : 0];
        const uint64_t kk = (ref < a.n_refs && lo <= d.n && k <= d.n - lo) ? k : 0;  // never past SA
        const IdxT *sa = reinterpret_cast<const IdxT *>(d.sa);
        for (uint64_t t = 0; t < kk; t++) {
            if (off + t < a.capacity) pos[off + t] = __ldg(sa + lo + t);
        }
        if (a.overflow != nullptr && off + kk > a.capacity) atomicOr(a.overflow, 1);
    }
}

}  // namespace

uint64_t locate_tiles(uint64_t n_q) { return (n_q + kTile - 1) / kTile; }

static_assert(kTile == 4096, "the static scratch below is sized for 4096-query tiles");
static_assert(kTile == (1ull << kLocateTileShift), "the search kernels sum kept counts per locate tile");

cudaError_t locate_static_partials(uint64_t **ptr, uint64_t *entries) {
    static std::mutex mu;
    static uint64_t *addr[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (addr[dev]) {
        // A device reset unloads the module; the array may then live at another
        // address.  The cached one is kept only while it is still device memory
        // of this device.
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, addr[dev]) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != dev) {
            cudaGetLastError();
            addr[dev] = nullptr;
        }
    }
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
    if (!L.presummed) tile_sums_kernel<<<(unsigned)tiles, kTileThreads, 0, s>>>(L.res, L.n_q, L.cap, L.partials);
    scan_partials_kernel<<<1, 1024, 0, s>>>(L.partials, tiles, L.base_in);
    if (L.width == 4)
        tile_gather_kernel<uint32_t><<<(unsigned)tiles, kTileThreads, 0, s>>>(L);
    else
        tile_gather_kernel<uint64_t><<<(unsigned)tiles, kTileThreads, 0, s>>>(L);
    return cudaGetLastError();
}

namespace {

// Copies the positions [*first, *last) of one chunk of a batch, clamped to
// the capacity, from the device array to the caller's host array (host
// memory the device can address).  The range is known only on the device.
template <typename IdxT>
__global__ void copy_positions_kernel(const uint64_t *__restrict__ first, const uint64_t *__restrict__ last,
                                      const IdxT *__restrict__ src, IdxT *dst, uint64_t capacity) {
    const uint64_t a = *first < capacity ? *first : capacity;
    const uint64_t b = *last < capacity ? *last : capacity;
    for (uint64_t i = a + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

}  // namespace

cudaError_t launch_copy_positions(const uint64_t *first, const uint64_t *last, const void *src, void *dst,
                                  uint32_t width, uint64_t capacity, cudaStream_t s) {
    const unsigned blocks = (unsigned)device_sm_count() / 2u + 1u;  // a few SMs: the link is the limit
    if (width == 4)
        copy_positions_kernel<uint32_t><<<blocks, 256, 0, s>>>(first, last, reinterpret_cast<const uint32_t *>(src),
                                                               reinterpret_cast<uint32_t *>(dst), capacity);
    else
        copy_positions_kernel<uint64_t><<<blocks, 256, 0, s>>>(first, last, reinterpret_cast<const uint64_t *>(src),
                                                               reinterpret_cast<uint64_t *>(dst), capacity);
    return cudaGetLastError();
}

}  // namespace sa
