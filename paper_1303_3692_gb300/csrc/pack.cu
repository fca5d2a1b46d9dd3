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

// Packs a whole query batch as one text (the layout of the reference) and
// records, per 32-base word, which bytes are not bases, so that the search
// reads any window of any query with one text_window and checks a query's
// validity from its own bytes only.  With a batch flag (dirty) a word's mask
// is stored only when it holds a non-base byte, and the flag is raised; the
// search then reads masks only for a batch whose flag is set, which the
// launcher packs again with every mask (only_if_dirty).  One thread per word; when the batch
// starts on a 16-byte boundary a full word is two 16-byte loads, so the reads
// are fully coalesced.  Words past the batch (padding) are zero.
__global__ void pack_batch_kernel(const uint8_t *__restrict__ ascii, uint64_t total, uint64_t nwords,
                                  uint64_t *__restrict__ tq, uint32_t *__restrict__ tv, bool aligned16, int *dirty,
                                  const int *only_if_dirty) {
    if (only_if_dirty != nullptr && *only_if_dirty == 0) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords + SA_TQ_PAD_WORDS; w += stride) {
        if (w >= nwords) {
            tq[w] = 0;
            tv[w] = 0;
            continue;
        }
        const uint64_t b0 = w * 32;
        uint64_t word;
        uint32_t bad = 0;
        if (aligned16 && b0 + 32 <= total) {
            const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(ascii + b0));
            const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(ascii + b0 + 16));
            const uint32_t v[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
            word = 0;
#pragma unroll
            for (int k = 0; k < 8; k++) word = (word << 8) | pack4_fast(v[k], &bad);
        } else {
            const uint64_t left = total - b0;
            word = pack_word(ascii, total, b0, left < 32 ? (uint32_t)left : 32u, &bad);
        }
        tq[w] = word;
        uint32_t mask = 0;
        if (bad) {  // rare: find which bytes are not bases
            for (uint32_t j = 0; j < 32 && b0 + j < total; j++)
                if (base_code(ascii[b0 + j]) > 3) mask |= 1u << j;
        }
        if (dirty == nullptr || mask != 0u) tv[w] = mask;
        if (mask != 0u && dirty != nullptr) atomicOr(dirty, 1);
    }
}

// The same for the reverse complement of the whole batch (the other strand):
// base i of the packed text is the complement of byte total - 1 - i, so query
// q's reverse complement is bases [total - qe, total - qa) of it.  Word w is
// packed from the 32 source bytes ending at total - 32 w, then its 2-bit codes
// are complemented (c -> 3 - c, i.e. every bit flipped) and put in reverse
// order; its validity mask is reversed the same way.
__global__ void pack_batch_rc_kernel(const uint8_t *__restrict__ ascii, uint64_t total, uint64_t nwords,
                                     uint64_t *__restrict__ tq, uint32_t *__restrict__ tv, int *dirty,
                                     const int *only_if_dirty) {
    if (only_if_dirty != nullptr && *only_if_dirty == 0) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords + SA_TQ_PAD_WORDS; w += stride) {
        if (w >= nwords) {
            tq[w] = 0;
            tv[w] = 0;
            continue;
        }
        const uint64_t b0 = w * 32;  // first base of the word in the reverse-complement text
        uint64_t word = 0;
        uint32_t mask = 0;
        if (b0 + 32 <= total) {
            const uint64_t src = total - b0 - 32;  // its 32 source bytes, in forward order
            uint32_t bad = 0;
            const uint64_t fwd = pack_word(ascii, total, src, 32u, &bad);
            const uint64_t flipped = __brevll(~fwd);  // complement, reverse the bit order
            // reversing the bits also swapped the two bits of every code: swap them back
            word = ((flipped >> 1) & 0x5555555555555555ull) | ((flipped & 0x5555555555555555ull) << 1);
            if (bad) {
                for (uint32_t j = 0; j < 32; j++)
                    if (base_code(ascii[src + 31 - j]) > 3) mask |= 1u << j;
            }
        } else {  // the last, partial word: bytes one at a time
            for (uint32_t j = 0; j < 32; j++) {
                uint32_t code = 0;
                if (b0 + j < total) {
                    const uint32_t c = base_code(ascii[total - 1 - b0 - j]);
                    if (c > 3) {
                        mask |= 1u << j;
                    } else {
                        code = 3u - c;
                    }
                }
                word = (word << 2) | code;
            }
        }
        tq[w] = word;
        if (dirty == nullptr || mask != 0u) tv[w] = mask;
        if (mask != 0u && dirty != nullptr) atomicOr(dirty, 1);
    }
}

cudaError_t launch_pack_batch(const SearchLaunch &L, uint64_t *tq, uint32_t *tv, cudaStream_t s) {
    const int threads = 256;
    const uint64_t want = (L.nwords + SA_TQ_PAD_WORDS + threads - 1) / threads;
    const uint64_t cap = (uint64_t)device_sm_count() * 8;
    const unsigned blocks = (unsigned)(want < cap ? want : cap);
    const bool aligned = ((uintptr_t)L.ascii & 15u) == 0;
    const uint8_t *ascii = reinterpret_cast<const uint8_t *>(L.ascii);
    // the forward packing, the reverse-complement one, or both (forward
    // first, the other from word nwords + SA_TQ_PAD_WORDS on) when each query
    // names its strand
    if (!L.revcomp || L.strand_bits)
        pack_batch_kernel<<<blocks, threads, 0, s>>>(ascii, L.total, L.nwords, tq, tv, aligned, L.batch_dirty,
                                                     nullptr);
    if (L.revcomp || L.strand_bits) {
        const uint64_t half = L.strand_bits ? L.nwords + SA_TQ_PAD_WORDS : 0;
        pack_batch_rc_kernel<<<blocks, threads, 0, s>>>(ascii, L.total, L.nwords, tq + half, tv + half,
                                                        L.batch_dirty, nullptr);
    }
    // With a batch flag the passes above store only the masks of words that
    // hold a non-base byte (the search reads no masks of a clean batch); a
    // batch that is not clean is packed again with every mask (these
    // launches return at once for a clean one).
    if (L.batch_dirty != nullptr) {
        if (!L.revcomp || L.strand_bits)
            pack_batch_kernel<<<blocks, threads, 0, s>>>(ascii, L.total, L.nwords, tq, tv, aligned, nullptr,
                                                         L.batch_dirty);
        if (L.revcomp || L.strand_bits) {
            const uint64_t half = L.strand_bits ? L.nwords + SA_TQ_PAD_WORDS : 0;
            pack_batch_rc_kernel<<<blocks, threads, 0, s>>>(ascii, L.total, L.nwords, tq + half, tv + half, nullptr,
                                                            L.batch_dirty);
        }
    }
    return cudaGetLastError();
}

}  // namespace sa
