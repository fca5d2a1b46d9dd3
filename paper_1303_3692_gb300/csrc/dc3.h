// dc3.h -- the host-side suffix-array construction of Section III (the
// difference cover modulo 3, DC3), shared by the C ABI entry point and the
// device build that uploads its result.  Plain C++: no CUDA types.
#pragma once

#include <cstdint>

namespace sa {

// Suffix array of n ASCII bases (A, C, G, T in either case) into sa[0..n),
// in the order of Table I.  Returns SA_OK, SA_ERR_BASE (a byte outside the
// alphabet; sa is then unspecified) or SA_ERR_NOMEM.  Requires 1 <= n < 2^32 - 1.
int dc3_suffix_array(const char *text, uint64_t n, uint32_t *sa);

}  // namespace sa
