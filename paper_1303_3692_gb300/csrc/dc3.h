// dc3.h -- the host-side suffix-array construction of Section III (the
// difference cover modulo 3, DC3), shared by the C ABI entry point and the
// index build that uploads its result.  Plain C++: no CUDA types.
#pragma once

#include <cstdint>

struct sa_index;

namespace sa {

// Builds idx's suffix array by dc3_suffix_array from host_text (host memory,
// idx->n bases) and uploads it on `stream` (a cudaStream_t), widening it on
// the device for 64-bit indexes.  Synchronous.  Defined in build.cu.
int build_suffix_array_host(::sa_index *idx, const char *host_text, void *stream);

// Suffix array of n ASCII bases (A, C, G, T in either case) into sa[0..n),
// in the order of Table I.  Returns SA_OK, SA_ERR_BASE (a byte outside the
// alphabet; sa is then unspecified) or SA_ERR_NOMEM.  Requires 1 <= n < 2^32 - 1.
int dc3_suffix_array(const char *text, uint64_t n, uint32_t *sa);

}  // namespace sa
