// pack.cu -- ASCII bases to the 2-bit big-endian layout (Section III alphabet).
#include "sa_internal.cuh"

namespace sa {

// Four ASCII bytes (little-endian in v) to four 2-bit codes in the low byte,
// first base in the top two bits.  Per byte, with u the case-folded byte:
// x = (u >> 1) & 3 is A0 C1 G3 T2 and c = x ^ (x >> 1) is A0 C1 G2 T3.  The
// codes sit at bits 0, 8, 16, 24; one multiply by 2^30 + 2^20 + 2^10 + 1
// moves them to bits 30, 28, 26, 24 without carries between the partial
// products.  The check rebuilds each letter from its code, 'A' + 2c + 2h +
// 11 (c & h) with h = c >> 1 (giving A, C, G, T for c = 0..3), and ORs any
// difference from u into *bad.
__device__ __forceinline__ uint32_t pack4_fast(uint32_t v, uint32_t *bad) {
    const uint32_t u = v & 0xDFDFDFDFu;
    const uint32_t x = (u >> 1) & 0x03030303u;
    const uint32_t h0 = (x >> 1) & 0x01010101u;
    const uint32_t c = x ^ h0;                     // per byte: A0 C1 G2 T3
    const uint32_t h = (c >> 1) & 0x01010101u;
    const uint32_t expect = 0x41414141u + 2u * c + 2u * h + 11u * (c & h);
    *bad |= u ^ expect;
    return (c * 0x40100401u) >> 24;
}

// One thread per packed word; words past the text (padding) are zero.
__global__ void pack_text_kernel(const uint8_t *__restrict__ ascii, uint64_t n, uint64_t *__restrict__ words,
                                 uint64_t nwords_padded, int *err_flag, bool aligned16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords_padded; w += stride) {
        const uint64_t b0 = w * 32;
        uint64_t word = 0;
        uint32_t bad = 0;
        if (b0 + 32 <= n && aligned16) {
            const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(ascii + b0));
            const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(ascii + b0 + 16));
            const uint32_t v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int k = 0; k < 8; k++) word = (word << 8) | pack4_fast(v[k], &bad);
        } else {
            for (int j = 0; j < 32; j++) {
                const uint64_t b = b0 + j;
                uint32_t code = 0;
                if (b < n) {
                    code = base_code(ascii[b]);
                    if (code > 3) {
                        bad |= 1u;
                        code = 0;
                    }
                }
                word = (word << 2) | code;
            }
        }
        words[w] = word;
        if (bad) atomicOr(err_flag, 1);
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

// Packs 32 ASCII bases starting at byte s of a (nb <= 32 bytes belong to the
// query; the rest pack as A).  When nine aligned 32-bit words around them lie
// inside [a, a + total) they are read and aligned with funnel shifts, and the
// bases past nb are masked to A afterwards; those bytes belong to the next
// query, which checks them itself.  Only the batch's last word takes the
// byte loop.
__device__ __forceinline__ uint64_t pack_word(const uint8_t *__restrict__ a, uint64_t total, uint64_t s,
                                              uint32_t nb, uint32_t *bad) {
    const uintptr_t lo_addr = ((uintptr_t)(a + s)) & ~(uintptr_t)3;
    uint64_t word = 0;
    if (lo_addr >= (uintptr_t)a && lo_addr + 36 <= (uintptr_t)(a + total)) {
        const uint32_t *p = reinterpret_cast<const uint32_t *>(lo_addr);
        const uint32_t sh = (uint32_t)(((uintptr_t)(a + s)) & 3u) * 8u;
        uint32_t v[9];
#pragma unroll
        for (int i = 0; i < 9; i++) v[i] = __ldg(p + i);
        uint32_t hi = 0, lo = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) hi = (hi << 8) | pack4_fast(__funnelshift_r(v[i], v[i + 1], sh), bad);
#pragma unroll
        for (int i = 4; i < 8; i++) lo = (lo << 8) | pack4_fast(__funnelshift_r(v[i], v[i + 1], sh), bad);
        word = ((uint64_t)hi << 32) | lo;
        if (nb < 32) word &= ~0ull << (64u - 2u * nb);
    } else {
        for (uint32_t j = 0; j < 32; j++) {
            uint32_t code = 0;
            if (j < nb) {
                code = base_code(a[s + j]);
                if (code > 3) {
                    *bad |= 1u;
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
// contiguous kilobyte.  The lane that packs a query's first word also writes
// the query's record for the search: the bracket from the reference's k-mer
// table when m >= k, else the whole range [-1, n).
__global__ void pack_queries_kernel(const __grid_constant__ SearchLaunch a, int *err_flag) {
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint8_t *ascii = reinterpret_cast<const uint8_t *>(a.ascii);
    uint32_t bad = 0;
    for (uint64_t q0 = warp * 32; q0 < a.n_q; q0 += nwarps * 32) {
        const uint64_t q = q0 + lane;
        uint64_t qa = 0, qe = 0;
        uint32_t words = 0, r = 0;
        if (q < a.n_q) {
            qa = __ldg(a.q_off + q) - a.first;
            qe = __ldg(a.q_off + q + 1) - a.first;
            r = a.q_ref ? __ldg(a.q_ref + q) : 0u;
            const bool range_ok = qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
            if (!range_ok) bad |= 1u;  // inconsistent offsets: the batch is reported invalid
            if (!range_ok || r >= a.n_refs) {
                a.meta[2 * q] = make_uint4(0u, 0u, kQueryInvalid, 0u);
                qa = qe = 0;
            } else if (qe == qa) {
                a.meta[2 * q] = make_uint4(0xFFFFFFFFu, (uint32_t)a.refs.r[r].n, 0u, 0u);
            } else {
                words = (uint32_t)((qe - qa + 31) >> 5);
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
            const uint64_t ai = __shfl_sync(0xFFFFFFFFu, qa, i);
            const uint64_t ei = __shfl_sync(0xFFFFFFFFu, qe, i);
            const uint32_t exi = __shfl_sync(0xFFFFFFFFu, excl, i);
            const uint32_t ri = __shfl_sync(0xFFFFFFFFu, r, i);
            if (t < W) {
                const uint32_t j = t - exi;
                const uint64_t s = ai + 32ull * j;
                const uint64_t left = ei - s;
                const uint32_t nb = left < 32 ? (uint32_t)left : 32u;
                const uint64_t slot = query_slot(ai, q0 + i);
                const uint64_t word = pack_word(ascii, a.total, s, nb, &bad);
                a.qwords[4 * slot + j] = word;
                uint64_t *mq = reinterpret_cast<uint64_t *>(a.meta + 2 * (q0 + i) + 1);
                if (j == 0) {
                    const RefDesc &d = a.refs.r[ri];
                    const uint32_t m = (uint32_t)(ei - ai);
                    uint32_t L = 0xFFFFFFFFu, R = (uint32_t)d.n;
                    if (d.kmer != nullptr && m >= d.kmer_k) {
                        const uint32_t x = (uint32_t)(word >> (64u - 2u * d.kmer_k));
                        L = __ldg(d.kmer + x) - 1u;
                        R = __ldg(d.kmer + x + 1);
                    }
                    a.meta[2 * (q0 + i)] = make_uint4(L, R, m, (uint32_t)slot);
                    mq[0] = word;
                    if (ei - ai <= 32) mq[1] = 0;
                } else if (j == 1) {
                    mq[1] = word;
                }
            }
        }
    }
    if (__any_sync(0xFFFFFFFFu, bad != 0) && lane == 0) atomicOr(err_flag, 1);
}

cudaError_t launch_pack_queries(const SearchLaunch &L, int *err_flag, cudaStream_t s) {
    const int threads = 256;
    const uint64_t warps_needed = (L.n_q + 31) / 32;
    const uint64_t cap = (uint64_t)device_sm_count() * 16;  // 16 blocks x 8 warps per SM
    uint64_t blocks = (warps_needed + 7) / 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    pack_queries_kernel<<<(unsigned)blocks, threads, 0, s>>>(L, err_flag);
    return cudaGetLastError();
}

}  // namespace sa
