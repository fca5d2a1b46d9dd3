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
// Every word goes to the query's 32-byte slots; the first two words and the
// validity are gathered in shared memory.  After the rounds each lane looks
// up its own query's bracket in the reference's k-mer table (when m >= k;
// else the bracket is [-1, n)) -- the 32 lookups of a warp in flight together
// -- and writes the query's whole 32-byte record in one coalesced store.  A query
// with a byte outside {A,C,G,T,a,c,g,t}, inconsistent offsets or an
// out-of-range reference id gets m = kQueryInvalid.
constexpr int kPackThreads = 256;

__global__ void __launch_bounds__(kPackThreads) pack_queries_kernel(const __grid_constant__ SearchLaunch a,
                                                                    int *err_flag) {
    __shared__ uint64_t s_w[kPackThreads / 32][32][2];
    __shared__ uint32_t s_bad[kPackThreads / 32][32];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned wib = threadIdx.x >> 5;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint8_t *ascii = reinterpret_cast<const uint8_t *>(a.ascii);
    bool any_bad = false;
    for (uint64_t q0 = warp * 32; q0 < a.n_q; q0 += nwarps * 32) {
        const uint64_t q = q0 + lane;
        uint64_t qa = 0, qe = 0;
        uint32_t words = 0, r = 0, m = kQueryInvalid;
        if (q < a.n_q) {
            qa = __ldg(a.q_off + q) - a.first;
            qe = __ldg(a.q_off + q + 1) - a.first;
            r = a.q_ref ? __ldg(a.q_ref + q) : 0u;
            const bool range_ok = qa <= qe && qe <= a.total && qe - qa < (1ull << 31);
            if (!range_ok) any_bad = true;
            if (range_ok && r < a.n_refs) {
                m = (uint32_t)(qe - qa);
                words = (m + 31) >> 5;
            } else {
                qa = qe = 0;
            }
        }
        s_w[wib][lane][0] = 0;
        s_w[wib][lane][1] = 0;
        s_bad[wib][lane] = 0;
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
            if (t < W) {
                const uint32_t j = t - exi;
                const uint64_t s = ai + 32ull * j;
                const uint64_t left = ei - s;
                const uint32_t nb = left < 32 ? (uint32_t)left : 32u;
                uint32_t bad = 0;
                const uint64_t word = pack_word(ascii, a.total, s, nb, &bad);
                a.qwords[4 * query_slot(ai, q0 + i) + j] = word;
                if (j < 2) s_w[wib][i][j] = word;
                if (bad) {
                    s_bad[wib][i] = 1;
                    any_bad = true;
                }
            }
        }
        __syncwarp();
        // Each lane brackets its own query from the k-mer table (the warp's 32
        // lookups in flight together) and writes the query's record.
        if (q < a.n_q) {
            const uint32_t mm = s_bad[wib][lane] ? kQueryInvalid : m;
            const uint64_t w0 = s_w[wib][lane][0], w1 = s_w[wib][lane][1];
            uint32_t L = 0xFFFFFFFFu, R = 0;
            if (m != kQueryInvalid) {
                const RefDesc &d = a.refs.r[r];
                R = (uint32_t)d.n;
                if (d.kmer != nullptr && m > 0 && m >= d.kmer_k) {
                    const uint32_t x = (uint32_t)(w0 >> (64u - 2u * d.kmer_k));
                    L = __ldg(d.kmer + x) - 1u;
                    R = __ldg(d.kmer + x + 1);
                }
            }
            a.meta[2 * q] = make_uint4(L, R, mm, (uint32_t)query_slot(qa, q));
            a.meta[2 * q + 1] = make_uint4((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1, (uint32_t)(w1 >> 32));
        }
        __syncwarp();
    }
    if (__any_sync(0xFFFFFFFFu, any_bad) && lane == 0) atomicOr(err_flag, 1);
}

cudaError_t launch_pack_queries(const SearchLaunch &L, int *err_flag, cudaStream_t s) {
    const int threads = kPackThreads;
    const uint64_t warps_needed = (L.n_q + 31) / 32;
    const uint64_t cap = (uint64_t)device_sm_count() * 16;  // 16 blocks x 8 warps per SM
    uint64_t blocks = (warps_needed + 7) / 8;
    if (blocks > cap) blocks = cap;
    if (blocks == 0) blocks = 1;
    pack_queries_kernel<<<(unsigned)blocks, threads, 0, s>>>(L, err_flag);
    return cudaGetLastError();
}

}  // namespace sa
