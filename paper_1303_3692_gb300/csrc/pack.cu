// pack.cu -- ASCII bases to the 2-bit big-endian layout (Section III alphabet).
#include "sa_internal.cuh"

namespace sa {

// Four ASCII bytes (little-endian in v) to four 2-bit codes in the low byte,
// first base in the top two bits; *ok is cleared if a byte is not a base.
__device__ __forceinline__ uint32_t pack4(uint32_t v, bool *ok) {
    const uint32_t u = v & 0xDFDFDFDFu;
    const uint32_t valid = __vcmpeq4(u, 0x41414141u) | __vcmpeq4(u, 0x43434343u) |
                           __vcmpeq4(u, 0x47474747u) | __vcmpeq4(u, 0x54545454u);
    *ok = *ok && valid == 0xFFFFFFFFu;
    const uint32_t x = (u >> 1) & 0x03030303u;
    const uint32_t c = x ^ ((x >> 1) & 0x01010101u);  // per byte: A0 C1 G2 T3
    return ((c & 0xFFu) << 6) | (((c >> 8) & 0xFFu) << 4) | (((c >> 16) & 0xFFu) << 2) | (c >> 24);
}

// One thread per packed word; words past the text (padding) are zero.
__global__ void pack_text_kernel(const uint8_t *__restrict__ ascii, uint64_t n, uint64_t *__restrict__ words,
                                 uint64_t nwords_padded, int *err_flag, bool aligned16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords_padded; w += stride) {
        const uint64_t b0 = w * 32;
        uint64_t word = 0;
        bool ok = true;
        if (b0 + 32 <= n && aligned16) {
            const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(ascii + b0));
            const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(ascii + b0 + 16));
            const uint32_t v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int k = 0; k < 8; k++) word = (word << 8) | pack4(v[k], &ok);
        } else {
            for (int j = 0; j < 32; j++) {
                const uint64_t b = b0 + j;
                uint32_t code = 0;
                if (b < n) {
                    code = base_code(ascii[b]);
                    if (code > 3) {
                        ok = false;
                        code = 0;
                    }
                }
                word = (word << 2) | code;
            }
        }
        words[w] = word;
        if (!ok) atomicOr(err_flag, 1);
    }
}

cudaError_t launch_pack_text(const char *ascii, uint64_t n, uint64_t *words, uint64_t nwords_padded,
                             int *err_flag, cudaStream_t s) {
    const int threads = 256;
    const uint64_t want = (nwords_padded + threads - 1) / threads;
    const int blocks = (int)(want < (uint64_t)device_sm_count() * 16 ? want : (uint64_t)device_sm_count() * 16);
    const bool aligned = ((uintptr_t)ascii & 15u) == 0;
    pack_text_kernel<<<blocks > 0 ? blocks : 1, threads, 0, s>>>(reinterpret_cast<const uint8_t *>(ascii), n,
                                                                 words, nwords_padded, err_flag, aligned);
    return cudaGetLastError();
}

// Packs 32 ASCII bases starting at byte s of a (nb <= 32 valid bytes; the
// rest pack as A).  The common case reads nine aligned 32-bit words inside
// [a, a + total) and aligns them with funnel shifts.
__device__ __forceinline__ uint64_t pack_word(const uint8_t *__restrict__ a, uint64_t total, uint64_t s,
                                              uint32_t nb, bool *ok) {
    const uintptr_t lo_addr = ((uintptr_t)(a + s)) & ~(uintptr_t)3;
    uint64_t word = 0;
    if (nb == 32 && lo_addr >= (uintptr_t)a && lo_addr + 36 <= (uintptr_t)(a + total)) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(lo_addr);
        const uint32_t sh = (uint32_t)(((uintptr_t)(a + s)) & 3u) * 8u;
        uint32_t v[9];
#pragma unroll
        for (int i = 0; i < 9; i++) v[i] = __ldg(p + i);
#pragma unroll
        for (int i = 0; i < 8; i++) word = (word << 8) | pack4(__funnelshift_r(v[i], v[i + 1], sh), ok);
    } else {
        for (uint32_t j = 0; j < 32; j++) {
            uint32_t code = 0;
            if (j < nb) {
                code = base_code(a[s + j]);
                if (code > 3) {
                    *ok = false;
                    code = 0;
                }
            }
            word = (word << 2) | code;
        }
    }
    return word;
}

// Each warp takes 32 consecutive queries (one per lane), scans their word
// counts, and then packs one output word per lane per round: a round covers
// 32 consecutive 32-base words of the batch, so the lanes read one
// contiguous kilobyte.  Query q's words start at ((q_off[q] - q_off[0]) >> 5) + q.
__global__ void pack_queries_kernel(const uint8_t *__restrict__ ascii, const uint64_t *__restrict__ q_off,
                                    uint64_t first, uint64_t total, uint64_t n_q, uint64_t *__restrict__ qwords,
                                    int *err_flag) {
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    bool ok = true;
    for (uint64_t q0 = warp * 32; q0 < n_q; q0 += nwarps * 32) {
        const uint64_t q = q0 + lane;
        uint64_t a = 0, e = 0;
        uint32_t words = 0;
        if (q < n_q) {
            a = __ldg(q_off + q) - first;
            e = __ldg(q_off + q + 1) - first;
            if (a > e || e > total || e - a >= (1ull << 31)) {
                ok = false;  // inconsistent offsets: reported, nothing read or written
                a = e = 0;
            } else {
                words = (uint32_t)((e - a + 31) >> 5);
            }
        }
        uint32_t incl = words;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        const uint32_t excl = incl - words;
        const uint32_t W = __shfl_sync(0xFFFFFFFFu, incl, 31);
        for (uint32_t base = 0; base < W; base += 32) {
            const uint32_t t = base + lane;
            // owner: the last lane whose first word is <= t
            uint32_t i = 0;
#pragma unroll
            for (uint32_t b = 16; b > 0; b >>= 1) {
                const uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, i + b);
                if (ex <= t) i += b;
            }
            const uint64_t ai = __shfl_sync(0xFFFFFFFFu, a, i);
            const uint64_t ei = __shfl_sync(0xFFFFFFFFu, e, i);
            const uint32_t exi = __shfl_sync(0xFFFFFFFFu, excl, i);
            if (t < W) {
                const uint32_t j = t - exi;
                const uint64_t s = ai + 32ull * j;
                const uint64_t left = ei - s;
                const uint32_t nb = left < 32 ? (uint32_t)left : 32u;
                qwords[(ai >> 5) + q0 + i + j] = pack_word(ascii, total, s, nb, &ok);
            }
        }
    }
    if (__any_sync(0xFFFFFFFFu, !ok) && lane == 0) atomicOr(err_flag, 1);
}

cudaError_t launch_pack_queries(const char *ascii, const uint64_t *q_off, uint64_t first, uint64_t total,
                                uint64_t n_q, uint64_t *qwords, int *err_flag, cudaStream_t s) {
    const int threads = 256;
    const uint64_t warps_needed = (n_q + 31) / 32;
    const uint64_t cap = (uint64_t)device_sm_count() * 16;  // 16 blocks x 8 warps per SM
    uint64_t blocks = (warps_needed + 7) / 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    pack_queries_kernel<<<(unsigned)blocks, threads, 0, s>>>(reinterpret_cast<const uint8_t *>(ascii), q_off,
                                                             first, total, n_q, qwords, err_flag);
    return cudaGetLastError();
}

}  // namespace sa
