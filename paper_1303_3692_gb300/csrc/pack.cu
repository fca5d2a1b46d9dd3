// pack.cu -- ASCII bases to the 2-bit big-endian layout (Section III alphabet).
#include "sa_internal.cuh"

namespace sa {

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

// Packs every query and writes its record for the search.  Each warp takes
// 32 consecutive queries (one per lane), scans their word counts, and then
// packs one output word per lane per round: a round covers 32 consecutive
// 32-base words of the batch, so the lanes read one contiguous kilobyte.
// Every word goes to the query's 32-byte slots; the lane that packs a
// query's first word also writes the first part of its record (the bracket
// from the reference's k-mer table when m >= k, else [-1, n); m; the slot)
// and the first two words go to the record's second half.  A query with a
// byte outside {A,C,G,T,a,c,g,t} gets qbad[q] = 1.
__global__ void pack_queries_kernel(const __grid_constant__ SearchLaunch a, int *err_flag) {
    const unsigned lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint8_t *ascii = reinterpret_cast<const uint8_t *>(a.ascii);
    bool any_bad = false;
    for (uint64_t q0 = warp * 32; q0 < a.n_q; q0 += nwarps * 32) {
        const uint64_t q = q0 + lane;
        uint64_t qa = 0, qe = 0;
        uint32_t words = 0, r = 0;
        if (q < a.n_q) {
            qa = __ldg(a.q_off + q) - a.first;
            qe = __ldg(a.q_off + q + 1) - a.first;
            r = a.q_ref ? __ldg(a.q_ref + q) : 0u;
            const bool range_ok = qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
            a.qbad[q] = 0;
            if (!range_ok) any_bad = true;  // inconsistent offsets: this query is invalid
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
        __syncwarp();
        for (uint32_t base = 0; base < W; base += 32) {
            const uint32_t t = base + lane;
            uint32_t i = 0;  // owner: the last lane whose first word is <= t
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
                uint32_t bad = 0;
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
                if (bad) {
                    a.qbad[q0 + i] = 1;
                    any_bad = true;
                }
            }
        }
    }
    if (__any_sync(0xFFFFFFFFu, any_bad) && lane == 0) atomicOr(err_flag, 1);
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
