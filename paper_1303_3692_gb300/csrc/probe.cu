// probe.cu -- the device's rate of dependent random reads (32 bytes, or up
// to 512 contiguous bytes), the ceiling of the search's probes (a probe is one such read into a table far
// larger than L2; its rate is set by the DRAM's row activations, not by its
// copy bandwidth).
#include "sa_internal.cuh"

namespace sa {

namespace {

// Every thread follows a chain of `steps` reads: the next index depends on
// the value just read, so each thread has exactly one read in flight.  One
// read is kSectors aligned, contiguous 32-byte sectors fetched by independent
// loads (the chain depends on all of them).
template <int kSectors>
__global__ void chase_kernel(const uint4 *__restrict__ buf, uint64_t n_rec, uint32_t steps, uint64_t seed,
                             uint32_t *sink) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t x = (tid + 1) * 0x9E3779B97F4A7C15ull ^ seed;
    uint32_t acc = 0;
    for (uint32_t i = 0; i < steps; i++) {
        x = x * 6364136223846793005ull + 1442695040888963407ull + acc;
        const uint64_t idx = __umul64hi(x, n_rec);  // < n_rec
        uint32_t a = 0;
#pragma unroll
        for (int j = 0; j < kSectors; j++) {
            uint4 lo, hi;
            ldg32(buf + 2 * (idx * kSectors + j), &lo, &hi);
            a ^= lo.x ^ hi.w;
        }
        acc = a & 1u;
    }
    // Practically never true, but the compiler cannot know it, so the whole
    // chain of reads stays live.
    if (x == seed) *sink = acc;
}

}  // namespace

}  // namespace sa

extern "C" int sa_random_read_rate_ex(uint64_t buffer_bytes, uint32_t threads_per_sm, uint32_t steps,
                                      uint32_t read_bytes, double *reads_per_s, void *stream) {
    using namespace sa;
    if (!reads_per_s || buffer_bytes < 4096 || steps == 0 || threads_per_sm < 32 || threads_per_sm > 2048 ||
        threads_per_sm % 32)
        return SA_ERR_ARG;
    if (read_bytes != 32 && read_bytes != 64 && read_bytes != 128 && read_bytes != 256 && read_bytes != 512)
        return SA_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t sectors = read_bytes / 32;
    const uint64_t n_rec = buffer_bytes / read_bytes;  // reads start on read_bytes boundaries
    uint4 *buf = nullptr;
    uint32_t *sink = nullptr;
    if (cudaMalloc(&buf, n_rec * read_bytes) != cudaSuccess) {
        cudaGetLastError();
        return SA_ERR_NOMEM;
    }
    if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(buf);
        return SA_ERR_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMemsetAsync(buf, 0x5A, n_rec * read_bytes, s);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    const uint32_t threads = threads_per_sm < 1024 ? threads_per_sm : 1024;
    const uint32_t blocks = (uint32_t)device_sm_count() * (threads_per_sm / threads);
    auto launch = [&](uint64_t seed) {
        switch (sectors) {
            case 1: chase_kernel<1><<<blocks, threads, 0, s>>>(buf, n_rec, steps, seed, sink); break;
            case 2: chase_kernel<2><<<blocks, threads, 0, s>>>(buf, n_rec, steps, seed, sink); break;
            case 4: chase_kernel<4><<<blocks, threads, 0, s>>>(buf, n_rec, steps, seed, sink); break;
            case 8: chase_kernel<8><<<blocks, threads, 0, s>>>(buf, n_rec, steps, seed, sink); break;
            default: chase_kernel<16><<<blocks, threads, 0, s>>>(buf, n_rec, steps, seed, sink); break;
        }
        return cudaGetLastError();
    };
    if (err == cudaSuccess) err = launch(1);  // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) err = launch(2);
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms > 0.f) *reads_per_s = (double)blocks * threads * steps / (ms * 1e-3);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(buf);
    return status_from_cuda(err);
}

extern "C" int sa_random_read_rate(uint64_t buffer_bytes, uint32_t threads_per_sm, uint32_t steps, double *reads_per_s,
                                   void *stream) {
    return sa_random_read_rate_ex(buffer_bytes, threads_per_sm, steps, 32, reads_per_s, stream);
}
