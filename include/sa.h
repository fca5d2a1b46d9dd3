/*
 * sa.h -- C ABI of libsa.so: batched exact matching of DNA queries against
 * references by binary search over their suffix arrays, on one NVIDIA GB300
 * (sm_103a).  Method: Liao et al., "Ultra-fast Multiple Genome Sequence
 * Matching Using GPU" (arXiv:1303.3692).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Alphabet (Section III): Sigma = {a,c,g,t}; upper and lower case are the
 *    same base; the order is A < C < G < T.  Any other byte makes the call
 *    fail with SA_ERR_BASE.
 *  - Suffix order (Section III, Table I): lexicographic, and a suffix that is
 *    a proper prefix of another sorts first.
 *  - Results are half-open: the paper's closed [LB, RB] (Section IV) is
 *    reported as lo = LB, hi = RB + 1, count = hi - lo.  A query that does not
 *    occur gets lo = hi = its insertion point and count = 0.  An empty query
 *    matches every suffix: [0, n).
 *  - Return value: SA_OK (0) or a negative SA_ERR_* code; sa_strerror() names
 *    it.  No C++ exception crosses this boundary.  Argument errors are
 *    detected before any work is queued.
 *  - Asynchrony: work is queued on the given CUDA stream (NULL = the legacy
 *    default stream) and the call returns without waiting for it, except
 *    where a function says otherwise.  Pointers may be device memory or host
 *    memory (pageable or pinned); host buffers are staged through device
 *    memory inside the call.  Output written to pinned host memory is valid
 *    once the stream completes; output to pageable host memory is valid when
 *    the call returns.
 *  - Ownership: the caller owns every buffer it passes; the library owns the
 *    sa_index and its device memory until sa_free().  Scratch device memory
 *    is taken from a library-private stream-ordered pool and returned on the
 *    same stream.
 *  - Threads: calls on distinct streams may run concurrently from different
 *    host threads.  An sa_index may be searched concurrently; sa_free must not
 *    race with any use of the index.
 *  - Devices: an index lives on the device that was current at sa_build /
 *    sa_load; later calls using it must run with that device current.
 */
#ifndef PAPER_1303_3692_GB300_SA_H
#define PAPER_1303_3692_GB300_SA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SA_OK 0
#define SA_ERR_ARG -1      /* invalid argument (null pointer, size, flag, ref id) */
#define SA_ERR_BASE -2     /* a byte outside {A,C,G,T,a,c,g,t} */
#define SA_ERR_NOMEM -3    /* device or host allocation failed */
#define SA_ERR_CUDA -4     /* a CUDA runtime call failed */
#define SA_ERR_TIMEOUT -5  /* a bounded device-side wait ran out */
#define SA_ERR_CAPACITY -6 /* an output buffer is too small */
#define SA_ERR_IO -7       /* file could not be opened, read or written */
#define SA_ERR_FORMAT -8   /* file is not an index, or its checksum does not match */

/* sa_build flags. */
#define SA_W32 0x1u     /* store the suffix array as uint32 (n < 2^32 - 1) */
#define SA_W64 0x2u     /* store the suffix array as uint64 */
#define SA_NO_KMER 0x4u /* build no k-mer table (see sa_build) */
/* build the suffix array on the host by the DC3 construction of Section III
 * (sa_suffix_array_host) and upload it, instead of prefix doubling on the
 * GPU; the rest of the index is built on the GPU either way */
#define SA_BUILD_HOST 0x8u
/* build the suffix array on the GPU by the DC3 construction of Section III
 * (the steps of sa_suffix_array_host, as data-parallel passes) instead of
 * prefix doubling; the same array either way */
#define SA_BUILD_DC3 0x10u
/* k of the k-mer table, 1..15, in bits 8-11; 0 there picks k automatically. */
#define SA_KMER_K(k) ((uint32_t)(k) << 8)

/* Opaque index: 2-bit packed reference, its suffix array and its sampled-key
 * table, resident in device memory. */
typedef struct sa_index sa_index;

/* One query's result (Section IV: the SA interval of the query), 32 bytes:
 * one aligned DRAM sector, so that a result written to a random slot is one
 * whole-sector store. */
typedef struct sa_result {
    uint64_t lo;    /* first suffix-array rank whose suffix has the query as prefix */
    uint64_t hi;    /* one past the last such rank (= RB + 1) */
    uint64_t count; /* hi - lo: occurrences of the query in the reference */
    uint64_t flags; /* SA_RESULT_* bits */
} sa_result;

/* sa_result.flags: the query could not be searched (lo = hi = count = all-ones). */
#define SA_RESULT_INVALID 0x1u
/* sa_result.flags, set by sa_search_locate: count > cap, so only the first cap
 * positions of the interval were located.  (sa_search_batch leaves it clear;
 * after a separate sa_locate the condition is count > cap.) */
#define SA_RESULT_TRUNCATED 0x2u

/* Tuning knobs of the search kernel; zero fields take the defaults.
 * The results never depend on them. */
typedef struct sa_search_params {
    uint32_t threads_per_block; /* 32..1024, multiple of 32 */
    uint32_t blocks_per_sm;     /* persistent CTAs per SM (at most 1024 threads per SM in all:
                                   larger requests are reduced to that) */
    uint32_t key_depth;         /* shared-memory key-table depth d (<= the index's) */
    uint32_t chunk;             /* queries a warp takes from the global counter at once */
    void *search_events[2];     /* optional cudaEvent_t pair, recorded on the stream right
                                   before and after the search kernel (kernel timing) */
    uint32_t flags;             /* SA_PARAM_Q_RANGE: q_first and q_total are given;
                                   SA_PARAM_REVERSE_COMPLEMENT: search the other strand */
    uint32_t front_probes;      /* probes per query in the one-thread-per-query first
                                   pass before a query joins the worklist of the
                                   persistent kernel, at most 64 (0: 1 when some
                                   index has more suffixes than k-mers, else 3) */
    uint64_t q_first;           /* q_offsets[0] */
    uint64_t q_total;           /* q_offsets[n_q] - q_offsets[0] */
    int32_t *device_status;     /* optional caller-owned int32 in device memory: at the end
                                   of the call's work on the stream the library writes the
                                   call's status there (see "Device status" below) */
    uint32_t reserved[2];
} sa_search_params;

/*
 * Device status.  A call whose outputs are device memory returns as soon as
 * its work is queued, so it cannot return what the kernels find.  Given
 * sa_search_params.device_status, the call queues one more one-thread kernel
 * that stores, in order of precedence:
 *   SA_ERR_TIMEOUT   a bounded device-side wait (the persistent kernel's copy
 *                    of the key tables into shared memory, 2 s) ran out; the
 *                    results of the queries that kernel was to finish are
 *                    then undefined;
 *   SA_ERR_BASE      some query holds a byte outside {A,C,G,T,a,c,g,t} or has
 *                    offsets outside the batch (its result is all-ones);
 *   SA_ERR_ARG       some query names a reference id >= n_refs (all-ones);
 *   SA_ERR_CAPACITY  (sa_search_locate only) out_pos was too small for the
 *                    positions: out_offsets[n_q] > out_pos_capacity;
 *   SA_OK            otherwise.
 * The word is valid once the stream has reached the end of the call.  With
 * host outputs the call returns the same status itself.
 */

/* sa_search_params.flags: the caller states q_offsets[0] and the batch's
 * total bases, so a call with device-resident offsets reads nothing back to
 * the host and does not synchronize. */
#define SA_PARAM_Q_RANGE 0x1u
/* sa_search_params.flags: search every query's reverse complement (the other
 * strand: bases in reverse order, A<->T and C<->G) instead of the query, with
 * the results the reverse-complemented queries would give.  The paper
 * searches the forward strand only; this flag is an extension. */
#define SA_PARAM_REVERSE_COMPLEMENT 0x2u
/* sa_search_params.flags, for testing the error path only: the persistent
 * kernel's bounded wait for its key tables gives up at once, as if its limit
 * had run out (the kernel still waits, bounded, for the copies it started
 * before it exits).  The call then reports SA_ERR_TIMEOUT and the results of
 * the queries that kernel was to finish are undefined. */
#define SA_PARAM_EXPIRE_WAITS 0x4u
/* sa_search_params.flags: the order in which the batch's queries are
 * searched (the results do not depend on it).  By default a call whose
 * indexes take more than 48 GB of device memory searches in k-mer order: the
 * queries are first bucketed by their first k bases, so that the random
 * reads in flight stay within a narrow slice of the index (random reads over
 * a wider footprint than the GPU's address translation covers run up to five
 * times slower); smaller indexes are searched in input order, the queries a
 * k-mer entry settles finishing in a one-thread-per-query first pass.  These
 * flags force one order (setting both is SA_ERR_ARG).  The default takes
 * k-mer order only for batches of at least 2^20 queries: a smaller batch is
 * in flight all at once whatever its order.  A batch of 2^30 queries or more
 * is always searched in input order.  K-mer order takes about 140 bytes of
 * scratch per query for the ordered list (room for every bucket's estimated
 * share and for queries the estimate missed). */
#define SA_PARAM_KMER_ORDER 0x8u
#define SA_PARAM_INPUT_ORDER 0x10u
/* sa_search_params.flags: each query names its strand -- bit 31 of q_ref[q]
 * set means search query q's reverse complement (as SA_PARAM_REVERSE_COMPLEMENT
 * does for a whole batch); the reference id is q_ref[q] & 0x7FFFFFFF.  q_ref
 * is then required, also with one index (ids 0), and the batch is packed in
 * both directions (twice the packed batch's scratch).  Not together with
 * SA_PARAM_REVERSE_COMPLEMENT (SA_ERR_ARG).  sa_locate ignores bit 31 of q_ref. */
#define SA_PARAM_STRAND_PER_QUERY 0x20u

/*
 * sa_build -- index one reference (Section III).
 *
 * Packs the bases 2 bits each (A=0, C=1, G=2, T=3, base 0 in the most
 * significant bits of each 64-bit word), builds the suffix array of the text
 * on the GPU by prefix doubling (radix sorts of rank pairs; the result is the
 * unique suffix array of Table I's definition) -- or, with SA_BUILD_HOST, on
 * the host by DC3 as Section III does -- and derives the structures
 * the search reads:
 *  - the key table kept in shared memory (first 64 bases of the suffixes at
 *    ranks floor((2p+1) n / 2^(l+1)), the top levels of the binary search);
 *  - one 32-byte record per rank (the first 112 bases of that suffix and its
 *    position), so that a probe reads one aligned sector;
 *  - unless SA_NO_KMER, the k-mer table: for each of the 4^k k-base
 *    strings x a 64-byte entry with lo = kmer[x] = number of suffixes that
 *    sort before x and hi = kmer[x + 1] (a query of m >= k bases whose first
 *    k bases are x lies strictly between ranks lo - 1 and hi), and the
 *    position and first 192 bases of the suffix at rank
 *    lo - 1 + (hi - lo + 1) / 2, the first pivot of the binary search over
 *    that bracket -- so one read brackets a query and makes its first probe.
 *    Automatic k: the largest k with 4^k <= 3n, in 1..15 (64 * 4^k bytes:
 *    17 GB at k = 14 for 10^8 bases, 69 GB at k = 15).
 * Device memory: about n/4 + (width + 32) n bytes + the k-mer table.
 *
 *  text   n bytes of bases, host or device memory.
 *  n      number of bases, 1 <= n < 2^32 - 1.
 *  flags  SA_W32 or SA_W64 (exactly one): element width of the suffix array;
 *         optionally SA_NO_KMER or SA_KMER_K(k), and SA_BUILD_HOST or
 *         SA_BUILD_DC3 (not both).
 *  stream CUDA stream (cudaStream_t) or NULL.
 *  out    receives the new index.
 *
 * Synchronous: returns after the index is complete (it synchronizes the
 * stream) so that SA_ERR_BASE can be reported.  Errors: SA_ERR_ARG, SA_ERR_BASE,
 * SA_ERR_NOMEM, SA_ERR_CUDA.  On error *out is NULL.
 */
int sa_build(const char *text, uint64_t n, uint32_t flags, void *stream, sa_index **out);

/*
 * sa_search_batch -- find the suffix-array interval of every query
 * (Section IV; Alg. 1 computes the same LB and RB).
 *
 *  refs       n_refs index handles (host array).
 *  n_refs     1..64; all indexes must have the same suffix-array width.
 *  q_bases    concatenated query bases (host or device).
 *  q_offsets  n_q + 1 uint64 offsets into q_bases, non-decreasing, q_offsets[0]
 *             may be non-zero; query i is q_bases[q_offsets[i] .. q_offsets[i+1]).
 *             Only the first and last entry are read on the host (with one
 *             small synchronous copy when the array is in device memory,
 *             unless sa_search_batch_ex is given SA_PARAM_Q_RANGE).
 *  q_ref      n_q reference ids (< n_refs), or NULL when n_refs == 1.
 *  n_q        number of queries, < 2^32 (0 is allowed and does nothing).
 *  out        n_q results (host or device; in device memory 32-byte aligned,
 *             since each result is stored as one 32-byte sector).
 *  stream     CUDA stream or NULL.
 *
 * The work runs as three kernels on the stream: the batch's bases are packed
 * 2 bits each beside a per-base validity mask; a one-thread-per-query pass
 * brackets each query of m >= k bases by the k-mer table and probes it up to
 * sa_search_params.front_probes times; a persistent kernel finishes the
 * queries that remain (and every query of an index without a k-mer table or
 * shorter than k).  Scratch device memory from the library pool: about
 * 12 * ceil(total / 32) + 64 n_q bytes (total = the batch's bases), plus the
 * staging copies of host inputs.
 *
 * A query that cannot be searched -- a byte outside {A,C,G,T,a,c,g,t}, an
 * out-of-range q_ref, or offsets inconsistent with the batch's range -- gets
 * lo = hi = count = UINT64_MAX and flags = SA_RESULT_INVALID; the other
 * queries are unaffected.  When the
 * output is in host memory the call also reports it: SA_ERR_BASE for a byte
 * or range problem, else SA_ERR_ARG for a reference id.
 *
 * Errors: SA_ERR_ARG, SA_ERR_BASE (see above), SA_ERR_NOMEM, SA_ERR_CUDA.
 */
int sa_search_batch(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                    const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q,
                    sa_result *out, void *stream);

/* sa_search_batch with explicit tuning knobs (params may be NULL). */
int sa_search_batch_ex(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                       const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q,
                       sa_result *out, void *stream, const sa_search_params *params);

/*
 * sa_search_batch_plain -- same contract and results as sa_search_batch, by
 * the paper's direct scheme (Section IV, Alg. 1): one thread per query, two
 * independent binary searches over the whole suffix array (the lower bound
 * LB, then the upper bound RB + 1), bases compared one at a time.  It is the
 * comparison point for the optimized kernel.
 */
int sa_search_batch_plain(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                          const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q,
                          sa_result *out, void *stream);

/*
 * sa_locate -- text positions of the matches (an extension; the paper
 * returns only [LB, RB]).
 *
 * For query i, writes the first k_i = min(res[i].count, cap) suffix-array
 * entries res[i].lo, res[i].lo + 1, ... (suffix-array order) to out_pos at
 * out_offsets[i]; out_offsets (n_q + 1 entries) is the exclusive prefix sum
 * of k_i and out_offsets[n_q] is the total.
 *
 *  refs, n_refs, q_ref   as for sa_search_batch (q_ref selects the index).
 *  res        n_q results of sa_search_batch (host or device).
 *  cap        positions kept per query (0 writes offsets of zeros).
 *  out_offsets n_q + 1 uint64 (host or device).
 *  out_pos    positions, element width = the indexes' suffix-array width
 *             (uint32 or uint64); may be NULL to compute only the offsets.
 *  out_pos_capacity  elements available in out_pos.  Positions whose slot
 *             is at or beyond it are not written.
 *
 * A query is truncated when res[i].count > cap: it then keeps the first cap
 * positions of its interval.  When out_pos is too small (out_offsets[n_q] >
 * out_pos_capacity) the positions that fit are written and, if out_offsets or
 * out_pos is host memory (the call then reads the total back and
 * synchronizes), the call returns SA_ERR_CAPACITY; with both in device memory
 * the call is asynchronous and the caller checks out_offsets[n_q] (or uses
 * sa_search_locate with a device status word).
 *
 * Errors: SA_ERR_ARG, SA_ERR_CAPACITY (see above), SA_ERR_NOMEM, SA_ERR_CUDA.
 */
int sa_locate(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref,
              const sa_result *res, uint64_t n_q, uint32_t cap, uint64_t *out_offsets,
              void *out_pos, uint64_t out_pos_capacity, void *stream);

/*
 * sa_search_locate -- sa_search_batch_ex followed by sa_locate on the same
 * stream in one call, with the same arguments and results as the two calls.
 *
 *  refs ... params  as for sa_search_batch_ex (out: n_q results).
 *  cap ... out_pos_capacity  as for sa_locate.
 *
 * Errors: as sa_search_batch (an invalid query gets the all-ones result and
 * no positions; the other queries are located) and sa_locate.  With
 * params->device_status the word also reports SA_ERR_CAPACITY when out_pos is
 * too small.
 */
int sa_search_locate(const sa_index *const *refs, uint32_t n_refs, const char *q_bases,
                     const uint64_t *q_offsets, const uint32_t *q_ref, uint64_t n_q,
                     sa_result *out, uint32_t cap, uint64_t *out_offsets, void *out_pos,
                     uint64_t out_pos_capacity, void *stream, const sa_search_params *params);

/* Largest n_q that sa_locate_noalloc accepts (its static scratch holds one
 * 8-byte partial sum per 4096 queries, plus one: 131,080 bytes). */
#define SA_LOCATE_NOALLOC_MAX_QUERIES (1ull << 26)

/*
 * sa_locate_noalloc -- sa_locate for callers that must not allocate device
 * memory.  The paper has no counterpart; this is a library service.
 *
 * Some callers cannot call cudaMalloc: an application whose device memory is
 * owned up front by another allocator (a framework's caching allocator or a
 * fixed arena sized at start-up), or a latency-critical loop where an
 * allocation could block on the device or fail under memory pressure.  This
 * entry point computes exactly what sa_locate computes but allocates nothing:
 * the scan's partial sums live in a file-scope __device__ array of
 * (SA_LOCATE_NOALLOC_MAX_QUERIES / 4096 + 1) uint64 that every device which
 * loads the library holds until the process exits.
 *
 *  Arguments are those of sa_locate, except that res, q_ref (if not NULL),
 *  out_offsets and out_pos (if not NULL) must all be device memory.
 *  n_q must be <= SA_LOCATE_NOALLOC_MAX_QUERIES.
 *
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Later calls check that the cached address is still device
 * memory of that device (one cudaPointerGetAttributes) and look it up again
 * if not: after cudaDeviceReset the module, and so the array, may move.  (A
 * reset also frees every index built before it.)  All calls share the one array and it keeps the last call's
 * contents (no call needs it to start at zero: every partial sum a call reads
 * is written earlier in the same call), so calls that overlap on the GPU race:
 * run them on one stream or order them with events.
 *
 * Errors: SA_ERR_CAPACITY if n_q exceeds the maximum, SA_ERR_ARG for a host
 * pointer or any argument sa_locate rejects, SA_ERR_CUDA.
 */
int sa_locate_noalloc(const sa_index *const *refs, uint32_t n_refs, const uint32_t *q_ref,
                      const sa_result *res, uint64_t n_q, uint32_t cap, uint64_t *out_offsets,
                      void *out_pos, uint64_t out_pos_capacity, void *stream);

/* Whether sa_search_batch_ex (or sa_search_locate) of n_q queries over these
 * indexes with these params (may be NULL) would search in k-mer order:
 * *kmer_order = 1, else 0 (see SA_PARAM_KMER_ORDER).  Errors: SA_ERR_ARG. */
int sa_search_order(const sa_index *const *refs, uint32_t n_refs, uint64_t n_q, const sa_search_params *params,
                    int *kmer_order);

/* Facts of the library's scratch pool on the current device: the bytes it
 * holds (reserved), the bytes allocated from it now (used) and the most ever
 * allocated at once since the last reset (used_high); reset_high != 0 then
 * resets that high-water mark.  Any output pointer may be NULL.  Lets a caller
 * see what scratch the library keeps, and check that a call allocated none.
 * Errors: SA_ERR_CUDA. */
int sa_scratch_info(uint64_t *reserved_bytes, uint64_t *used_bytes, uint64_t *used_high_bytes, int reset_high);

/* Writes the index (header, packed text, suffix array, key table and a
 * 64-bit FNV-1a checksum) to path.  Synchronous.  SA_ERR_IO on failure. */
int sa_save(const sa_index *idx, const char *path, void *stream);

/* Reads an index written by sa_save onto the current device.  Synchronous.
 * SA_ERR_IO, SA_ERR_FORMAT (bad magic, version or checksum), SA_ERR_NOMEM. */
int sa_load(const char *path, void *stream, sa_index **out);

/* Size facts of an index; any output pointer may be NULL.  kmer_k is 0 when
 * the index has no k-mer table. */
int sa_index_info(const sa_index *idx, uint64_t *n, uint32_t *width, uint32_t *key_depth,
                  uint32_t *kmer_k, uint64_t *device_bytes);

/*
 * sa_random_read_rate -- measures the device's rate of dependent random
 * 32-byte reads, the ceiling of the search's probes: threads_per_sm threads
 * per SM each follow a chain of `steps` reads, each read's address derived
 * from the value of the one before, over a buffer of buffer_bytes (allocated
 * and freed by the call; make it far larger than L2).  *reads_per_s receives
 * the reads completed per second.  Synchronous.
 *
 * Errors: SA_ERR_ARG (buffer_bytes < 4096, steps == 0, threads_per_sm not a
 * multiple of 32 in 32..2048), SA_ERR_NOMEM, SA_ERR_CUDA.
 */
int sa_random_read_rate(uint64_t buffer_bytes, uint32_t threads_per_sm, uint32_t steps, double *reads_per_s,
                        void *stream);

/* sa_random_read_rate with the size of one read: read_bytes (32, 64, 128,
 * 256 or 512) contiguous bytes starting on a read_bytes boundary, fetched as
 * independent 32-byte loads on which the next address depends.  Whether a
 * wider read costs one DRAM row activation or several decides how much a
 * search gains from wider nodes.  *reads_per_s counts reads, not sectors.
 * Errors: as sa_random_read_rate, and SA_ERR_ARG for any other read_bytes. */
int sa_random_read_rate_ex(uint64_t buffer_bytes, uint32_t threads_per_sm, uint32_t steps, uint32_t read_bytes,
                           double *reads_per_s, void *stream);

/* Copies the k-mer table's counts kmer[x] (4^k + 1 uint32, the last = n) to
 * dst (host or device; a host copy synchronizes the stream).  SA_ERR_ARG if
 * the index has none. */
int sa_copy_kmer_table(const sa_index *idx, void *dst, void *stream);

/* Copies the suffix array (n elements of the index's width) to dst (host or
 * device).  Asynchronous on stream for device/pinned dst. */
int sa_copy_suffix_array(const sa_index *idx, void *dst, void *stream);

/*
 * sa_suffix_array_host -- the suffix array of a text by the difference cover
 * modulo 3 (DC3, Section III: sort the suffixes at positions i mod 3 != 0 by
 * their leading triples, recursing on the string of triple ranks when two
 * coincide (Table II ranks them); order the suffixes at i mod 3 == 0 by their
 * first base and the rank of the next sample suffix; merge the two lists).
 * Runs on the host CPU, single-threaded, in O(n) time; needs no GPU.
 *
 *  text   n ASCII bases (A, C, G, T, either case), host memory.
 *  n      1 <= n < 2^32 - 1.
 *  width  4 or 8: element width of sa.
 *  sa     caller-owned host buffer of n elements: receives the suffix array in
 *         the order of Table I (a suffix that is a proper prefix of another
 *         sorts first).
 *
 * Errors: SA_ERR_ARG, SA_ERR_BASE (a byte outside the alphabet; sa is then
 * unspecified), SA_ERR_NOMEM (host memory: up to about 17 n bytes besides sa,
 * and 4 n more for width 8).
 */
int sa_suffix_array_host(const char *text, uint64_t n, uint32_t width, void *sa);

/*
 * sa_suffix_array_gpu -- the suffix array of a text, built on the GPU into a
 * caller-owned device buffer (no index): by prefix doubling, or with
 * SA_BUILD_DC3 in flags by the DC3 construction of Section III.
 *
 *  text   n bases (A, C, G, T, either case), host or device memory.
 *  n      1 <= n < 2^32 - 1.
 *  width  4 or 8: element width of sa.
 *  flags  0 or SA_BUILD_DC3.
 *  sa     device buffer of n elements (Table I order).
 *  stream CUDA stream or NULL.  Synchronous.
 *
 * Scratch comes from the library's pool: about 12 n bytes (prefix doubling
 * 46 n) besides sa.  Errors: SA_ERR_ARG, SA_ERR_BASE, SA_ERR_NOMEM, SA_ERR_CUDA.
 */
int sa_suffix_array_gpu(const char *text, uint64_t n, uint32_t width, uint32_t flags, void *sa, void *stream);

/*
 * The suffix tree (Section III), flattened for the GPU: the paper's
 * comparison index (Table V times a suffix-tree search beside the
 * suffix-array one).  Built from an index's suffix array and an LCP array
 * (computed on the GPU) by the bottom-up traversal of LCP intervals on the
 * host; one 32-byte record per internal node {first rank, last rank, string
 * depth, a text position of its label, a child per base}, leaves being single
 * ranks.  About 32 bytes of device memory per base.  For contrast: the
 * suffix-array search is the product path.
 */
typedef struct sa_stree sa_stree;

/* Builds the tree of idx's text.  Synchronous; the tree refers to idx, which
 * must outlive it.  Host memory about 45 n bytes during the build.  Errors:
 * SA_ERR_ARG, SA_ERR_NOMEM, SA_ERR_CUDA. */
int sa_stree_build(const sa_index *idx, void *stream, sa_stree **out);

/* The interval of every query by descending the tree, one GPU thread per
 * query: the same results as sa_search_batch (Section IV's interval; misses at
 * their insertion point; an invalid query all-ones with SA_RESULT_INVALID).
 * q_bases, q_offsets (n_q + 1) and out (32-byte aligned) in device memory.
 * Reads q_offsets[0] and q_offsets[n_q] back (one small synchronous copy).
 * Errors: SA_ERR_ARG, SA_ERR_NOMEM, SA_ERR_CUDA. */
int sa_stree_search(const sa_stree *t, const char *q_bases, const uint64_t *q_offsets, uint64_t n_q, sa_result *out,
                    void *stream);

/* Internal nodes and device bytes of a tree; either pointer may be NULL. */
int sa_stree_info(const sa_stree *t, uint64_t *nodes, uint64_t *device_bytes);

/* Releases the tree (synchronizes the device first); not its index. */
void sa_stree_free(sa_stree *t);

/* Releases the index and its device memory (synchronizes the device first). */
void sa_free(sa_index *idx);

/* Static English text for a status code. */
const char *sa_strerror(int status);

/* Library version, e.g. 0x000100 for 0.1.0. */
uint32_t sa_version(void);

#ifdef __cplusplus
}
#endif

#endif
