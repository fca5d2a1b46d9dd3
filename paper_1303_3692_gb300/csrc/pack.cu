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

// One warp per query: each step packs 128 bases, 4 per lane; the 8 lanes of
// an octet OR their bytes into one 32-base word, written by the octet's
// first lane.  Query q's words start at ((q_off[q] - q_off[0]) >> 5) + q.
__global__ void pack_queries_kernel(const uint8_t *__restrict__ ascii, const uint64_t *__restrict__ q_off,
                                    uint64_t first, uint64_t total, uint64_t n_q, uint64_t *__restrict__ qwords,
                                    int *err_flag) {
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    bool ok = true;
    for (uint64_t q = warp; q < n_q; q += nwarps) {
        const uint64_t a = __ldg(q_off + q) - first;
        const uint64_t e = __ldg(q_off + q + 1) - first;
        if (a > e || e > total) {  // inconsistent offsets: reported, nothing read or written
            ok = false;
            continue;
        }
        const uint64_t m = e - a;
        uint64_t *dst = qwords + (a >> 5) + q;
        for (uint64_t base = 0; base < m; base += 128) {
            const uint64_t b = a + base + 4u * lane;
            uint32_t v = 0x41414141u;  // bases past the end pack as A (code 0)
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (b + k < e) {
                    const uint32_t c = ascii[b + k];
                    v = (v & ~(0xFFu << (8 * k))) | (c << (8 * k));
                }
            }
            const uint64_t part = (uint64_t)pack4(v, &ok) << (56u - 8u * (lane & 7u));
            uint64_t word = part;
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
            word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
            const uint64_t wi = (base >> 5) + (lane >> 3);
            if ((lane & 7u) == 0 && wi * 32 < m) dst[wi] = word;
        }
    }
    if (__any_sync(0xFFFFFFFFu, !ok) && lane == 0) atomicOr(err_flag, 1);
}

cudaError_t launch_pack_queries(const char *ascii, const uint64_t *q_off, uint64_t first, uint64_t total,
                                uint64_t n_q, uint64_t *qwords, int *err_flag, cudaStream_t s) {
    const int threads = 256;
    const uint64_t warps_needed = n_q;
    const uint64_t cap = (uint64_t)device_sm_count() * 64;  // 8 blocks x 8 warps per SM
    uint64_t blocks = (warps_needed + 7) / 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    pack_queries_kernel<<<(unsigned)blocks, threads, 0, s>>>(reinterpret_cast<const uint8_t *>(ascii), q_off,
                                                             first, total, n_q, qwords, err_flag);
    return cudaGetLastError();
}

}  // namespace sa
