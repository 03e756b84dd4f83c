/*
 * leco.h — C ABI of the GB300 LeCo library (libleco.so).
 *
 * LeCo (Liu, Zeng & Zhang, "LeCo: Lightweight Compression via Learning Serial Correlations")
 * compresses an integer column by splitting it into partitions (§3.2), fitting one regression
 * model per partition (§3.1: constant = FOR, linear, or a polynomial of degree <= 3 chosen per
 * partition) and bit-packing the residuals ("deltas")
 * at a fixed width per partition (§3.3). This library runs encode, full decode, range decode,
 * batched point lookups and a fused filter + sum scan on one CUDA GPU (sm_103a).
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers on the current CUDA device; host_* are host pointers.
 *    The caller owns every buffer it passes in or out. The library owns the column (records,
 *    residual words, partition starts, decode table and status word), allocated on the device
 *    that is current when the column is created.
 *  - Calls are stream-ordered on `stream` (a cudaStream_t; NULL = the legacy default stream) and
 *    return before the GPU work completes, unless documented otherwise. Argument errors that the
 *    host can see are returned synchronously and then nothing is enqueued.
 *  - Device-side errors (an index >= n in a lookup) do not fail the call: the affected output
 *    slot gets 0 and the column's status word records the error; leco_sync() reports it.
 *  - A column is immutable after creation, so concurrent reads on different streams are safe.
 *  - n = 0 is valid: an empty column; decodes write nothing and sums are zero.
 *  - Values are unsigned 32- or 64-bit integers. Filter bounds compare as unsigned.
 *
 * Stored format (§3.3 storage format, with this library's readings):
 *  - One 32-byte record per partition: {double theta0, double theta1, uint64 start, uint64 word3}
 *    with word3 = bit offset (bits 0..47) | width b (48..54) | grid exponent s (55..61, two's
 *    complement) | exact flag (62) | polynomial flag (63).
 *  - Residuals: zigzag-coded, b bits each, packed LSB-first into one stream of little-endian
 *    64-bit words shared by all partitions; partition p starts at its bit offset, offsets dense.
 *    The stream carries at least two zero padding words and is a multiple of 16 bytes.
 *  - Value at local index i' of a partition: pred(i') + unzigzag(field) mod 2^64 (truncated to
 *    32 bits for 32-bit columns), with pred(i') = floor(fl(fl(theta1 * i') + theta0)) in IEEE
 *    binary64, one rounding per operation (no FMA), NaN -> 0 and saturation to int64 (§3.3
 *    decoder). When the exact flag is set the encoder guarantees that this equals
 *    (A + B i') >> s with the integers A = theta0 * 2^s, B = theta1 * 2^s (s < 0: no shift), which
 *    is what the device evaluates.
 *  - Polynomial partitions (flag 63; LECO_MODEL_POLY): theta0 = theta1 = 0, exact = 0, s = 0, and
 *    the partition's bits start with five 64-bit words T, K1, K2, K3 (two's complement) and
 *    E = s1 | s2 << 8 | s3 << 16 (each s_j in 0..62), followed by its residuals (residual i' at
 *    offset + 320 + b i'). With N the partition length, x' = 2 i' - (N - 1) and the Gram
 *    polynomials p1 = x', p2 = 3 x'^2 - (N^2 - 1), p3 = 5 x'^3 - (3 N^2 - 7) x', the prediction is
 *    pred(i') = T + floor(sum_j K_j p_j(i') 2^-s_j) mod 2^64, evaluated exactly in integers.
 *    A polynomial partition holds 64 .. 16384 values.
 */
#ifndef LECO_H
#define LECO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* leco_stream_t; /* identical to cudaStream_t */

typedef enum {
  LECO_OK = 0,
  LECO_ERR_INVALID_ARG = 1, /* a NULL, size or enum argument the call cannot accept */
  LECO_ERR_OOM = 2,         /* device or host allocation failed */
  LECO_ERR_INDEX_RANGE = 3, /* a lookup index was >= n (reported by leco_sync) */
  LECO_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  LECO_ERR_CORRUPT = 5,     /* a serialized blob failed validation */
  LECO_ERR_TIMEOUT = 6,     /* a bounded device wait gave up */
  LECO_ERR_BUDGET = 7       /* a server admission would exceed its memory budget */
} leco_status;

typedef enum { LECO_U32 = 0, LECO_U64 = 1 } leco_dtype;

/* §3.1 model family members built here: constant (FOR, §2), linear, and the polynomial model:
 * each partition takes whichever of constant, linear, quadratic and cubic (least squares on the
 * Gram polynomials, coefficients on binary grids) gives it the smallest exact size (record and
 * coefficient bits + len * b; ties to the simpler model). Variable partitioning and the
 * partition-size search size partitions with the linear model under LECO_MODEL_POLY. */
typedef enum { LECO_MODEL_CONSTANT = 0, LECO_MODEL_LINEAR = 1, LECO_MODEL_POLY = 2 } leco_model;

typedef enum { LECO_PART_FIXED = 0, LECO_PART_VAR = 1, LECO_PART_AUTO = 2, LECO_PART_VAR_SEEDED = 3 } leco_part_kind;

/* Partition policy (§3.2). Fixed: partition j = positions [j L, (j+1) L) (§3.2.1), part_size = L
 * (1 .. 2^24). Variable: split + merge (§3.2.2); part_size caps a partition's length (1 .. 2^24,
 * 0 = 2^24); tau in [0, 1] is the split threshold coefficient (C <= tau * S_M with S_M = 256 bits,
 * one record). Auto: fixed partitions whose size leco_search_partition_size picks (§3.2.1) over
 * 1 .. part_size (0 = 10000, at most 16384) from a 1% sample with seed 0. Variable seeded: as
 * variable, but each 65536-value chunk's split starts at the chunk's smoothest point (§3.2.2,
 * selecting good starting positions: the first window of three values whose second-order delta has
 * the shortest zigzag code) and grows partitions from there in both directions (the backward
 * direction with the same greedy rule on the values read backwards); the column is a variable
 * partition column. */
typedef struct {
  int32_t kind;       /* leco_part_kind */
  uint32_t part_size; /* fixed: L; variable: length cap */
  double tau;         /* variable only */
} leco_partition_policy;

typedef struct leco_column leco_column; /* opaque, device resident, immutable */

/* count and sum of the selected values; the sum is exact modulo 2^128 */
typedef struct {
  uint64_t count;
  uint64_t sum_lo;
  uint64_t sum_hi;
} leco_sum_result;

typedef struct {
  uint64_t n;              /* values */
  uint64_t partitions;     /* m */
  uint64_t record_bytes;   /* 32 m */
  uint64_t residual_bytes; /* 8 * padded word count */
  uint64_t total_bytes;    /* record_bytes + residual_bytes (+ 8 (m+1) start index for var) */
  double ratio;            /* total_bytes / (n * value bytes); 0 for n = 0 */
  int32_t dtype;           /* leco_dtype */
  int32_t kind;            /* leco_part_kind */
  int32_t model;           /* leco_model */
  uint32_t part_size;      /* fixed L (0 for variable) */
  uint64_t residual_bits;  /* bits of the stream: sum over partitions of len * b, plus 320 per
                              polynomial partition (its coefficient block) */
  uint64_t device_bytes;   /* bytes the column holds on the device */
} leco_stats;

/* Filter flags; every mode returns the identical result.
 * 0: scan every residual word of the column; each 32-value group is first bounded by its model
 *    (prediction at both ends +- the residual range of width b) and decoded only if it can meet
 *    [lo, hi] (groups certainly inside are summed without the compare).
 * LECO_FILTER_PRUNE: additionally skip reading the residuals of 2048-position tiles whose
 *    partitions' model bounds all miss [lo, hi] (the model-bound pruning of §5.1).
 * LECO_FILTER_DECODE_ALL: decode and compare every value (no group bounds); a diagnostic mode. */
#define LECO_FILTER_PRUNE 1u
#define LECO_FILTER_DECODE_ALL 2u

/* ------------------------------------------------------------------------------------------ */
/* Library */

/* Human-readable name of a status code; never NULL. Library plumbing; the paper has no counterpart. */
const char* leco_status_string(leco_status s);

/* ABI version (major * 10000 + minor * 100 + patch). Library plumbing; the paper has no counterpart. */
uint32_t leco_version(void);

/* ------------------------------------------------------------------------------------------ */
/* Encode (§3: Partitioner -> Regressor -> Encoder)
 *
 * d_values: n values of `dtype` (4 or 8 bytes each, contiguous) on the device, caller-owned, read
 * only. policy: fixed, variable or auto partitions. model: constant, linear or polynomial. On
 * success *out receives a new column (free with leco_column_free). The call synchronizes `stream` once (to size the
 * residual stream) and returns with the column's encode enqueued on `stream`.
 * Errors: INVALID_ARG (NULL out, NULL d_values with n > 0, part_size out of range, tau outside
 * [0,1], bad enum), OOM, CUDA. */
leco_status leco_encode(const void* d_values, uint64_t n, leco_dtype dtype,
                        leco_partition_policy policy, leco_model model, leco_stream_t stream,
                        leco_column** out);

/* Variable-length partitioning only (§3.2.2): split + merge on the device. d_starts_out receives
 * m+1 uint64 partition starts (the last is n) and must hold n+1 entries; *m_out = m. Synchronizes
 * `stream` once per merge round. Errors as leco_encode. */
leco_status leco_var_partition(const void* d_values, uint64_t n, leco_dtype dtype,
                               leco_partition_policy policy, leco_model model,
                               uint64_t* d_starts_out, uint64_t* m_out, leco_stream_t stream);

/* Encode with caller-chosen partition starts (§3.2: any partitioning the Partitioner hands over; §3.1
 * fit and §3.3 packing per partition as in leco_encode). d_starts: m+1 uint64 on the device,
 * caller-owned, read only: starts[0] = 0, starts[m] = n, strictly increasing, each partition at most
 * 2^24 long. The column is a variable partition column. Errors as leco_encode. */
leco_status leco_encode_with_starts(const void* d_values, uint64_t n, leco_dtype dtype,
                                    const uint64_t* d_starts, uint64_t m, leco_model model,
                                    leco_stream_t stream, leco_column** out);

/* Fixed-partition encode that allocates no device memory (the paper has no counterpart: this is
 * for callers that cannot call cudaMalloc, e.g. an engine whose device memory is all reserved by
 * its own pool, or a path that cannot afford an allocation's implicit synchronization).
 * Same records and residual words as leco_encode with policy fixed(L), written to caller buffers:
 *   d_values   n values of dtype on the device (read only);
 *   d_records  ceil(n / L) * 32 bytes on the device (the 32-byte records described above);
 *   d_words    words_cap * 8 bytes on the device (the residual stream, padding included);
 *   nwords_out host; receives the stream's word count, also when words_cap is too small.
 * Scratch lives in a fixed 12.6 MB __device__ array that every GPU loading the library holds
 * until exit; ceil(n / L) must not exceed 2^18 (INVALID_ARG otherwise). The first call on a
 * device looks up that array's device address; with CUDA's lazy module loading (the default) that
 * first call is also when the driver loads the encode kernels and creates the array, a driver
 * allocation of its own: make the first call on each device before any stream capture and before
 * the caller's own pool reserves the device's memory. All calls on a device share the array, so
 * calls whose GPU work overlaps (e.g. on different streams) race; nothing of it needs clearing
 * between calls. The call synchronizes `stream` twice: once to size the stream, and once at the
 * end to read back whether a staging copy of the packer gave up (then LECO_ERR_TIMEOUT: the words
 * are incomplete). INVALID_ARG when words_cap < *nwords_out (nothing packed then) or for
 * LECO_MODEL_POLY (constant and linear only), CUDA on a runtime failure. No cudaMalloc, cudaFree
 * or allocating library routine is called. */
leco_status leco_encode_fixed_noalloc(const void* d_values, uint64_t n, leco_dtype dtype, uint32_t L,
                                      leco_model model, void* d_records, void* d_words,
                                      uint64_t words_cap, uint64_t* nwords_out,
                                      leco_stream_t stream);

/* ------------------------------------------------------------------------------------------ */
/* Decode (§3.3 Decoder)
 *
 * Full decompression: d_out receives all n values (n * value bytes, caller-owned, device). */
leco_status leco_decode_all(const leco_column* col, void* d_out, leco_stream_t stream);

/* Range decompression (§3.3 Decoder) of positions [begin, begin + count): d_out receives count
 * values (count * value bytes, caller-owned, device). Errors: INVALID_ARG if begin + count > n. */
leco_status leco_decode_range(const leco_column* col, uint64_t begin, uint64_t count, void* d_out,
                              leco_stream_t stream);

/* Batched point lookups (§3.3 Decoder, random access; §4.3.2): d_out[q] = value at position d_idx[q]
 * for q < k (input order, duplicates allowed). d_idx: k uint64 on the device; d_out: k values of the
 * column's width on the device; both caller-owned. Fixed partitions use j = i / L; variable
 * partitions a search over the starts. An index >= n writes 0 and sets LECO_ERR_INDEX_RANGE in the
 * column status (see leco_sync). */
leco_status leco_random_access(const leco_column* col, const uint64_t* d_idx, uint64_t k,
                               void* d_out, leco_stream_t stream);

/* Fused filter + aggregate (the filter of §5.1.1, with its sum): count and sum of the values v with
 * lo <= v <= hi (unsigned, inclusive), never materialising the decoded column. d_out: one
 * leco_sum_result on the device, caller-owned, overwritten. lo > hi gives {0, 0, 0}. flags: any
 * combination of LECO_FILTER_PRUNE and LECO_FILTER_DECODE_ALL (the result is the same). Errors:
 * INVALID_ARG (NULL, unknown flag bits), CUDA. */
leco_status leco_filter_sum(const leco_column* col, uint64_t lo, uint64_t hi, uint32_t flags,
                            leco_sum_result* d_out, leco_stream_t stream);

/* Synchronize `stream`, then return the first device-side error recorded on the column since the
 * last leco_sync (and clear it), else LECO_OK; a failed synchronization returns LECO_ERR_CUDA.
 * Error reporting of this library; the paper has no counterpart. */
leco_status leco_sync(const leco_column* col, leco_stream_t stream);

/* Fixed partition-size search (§3.2.1): sample k = max(1, floor(sample_frac n / max_len))
 * subsequences of max_len values (starts SplitMix64(seed + i) mod (n - max_len + 1); a column of at
 * most max_len values is its own sample), then search L in 1 .. max_len for the smallest compressed
 * size of the sample under fixed partitions: an exponential phase over powers of two that ends after
 * the first size above its predecessor's, then a back search with halving steps, stopping when a move
 * gains less than 0.01 %. d_values: n values of dtype (device). max_len: 1 .. 16384 (0 = 10000);
 * sample_frac in (0, 1] (0 = 0.01). Writes the size to *best_L and, when non-NULL, the sample's size
 * in bits at that L to *best_bits and the number of sizes evaluated to *evals. Synchronizes `stream`
 * once per size evaluated. Errors: INVALID_ARG, OOM, CUDA. */
leco_status leco_search_partition_size(const void* d_values, uint64_t n, leco_dtype dtype, leco_model model,
                                       uint32_t max_len, double sample_frac, uint64_t seed, leco_stream_t stream,
                                       uint32_t* best_L, uint64_t* best_bits, uint64_t* evals);

/* Failure-detection self-test: one kernel waits on a shared-memory barrier that nothing completes,
 * with the same bounded wait the scan and pack kernels use, limited to limit_us microseconds
 * (1 .. 1000000). Returns LECO_ERR_TIMEOUT when the wait gave up and reported it (the expected
 * outcome: the device stays usable), LECO_OK if the barrier completed, INVALID_ARG or CUDA on
 * errors. Synchronizes `stream`. A systems facility; the paper has no counterpart. */
leco_status leco_selftest_wait_timeout(uint32_t limit_us, leco_stream_t stream);

/* Execution-unit throughput probe (a systems facility; the paper has no counterpart): runs many
 * independent chains of one kind of operation on every SM of the current device and returns the
 * measured rate in *ops_per_s. kind 0: 32-bit integer shift, xor and add (x = (x ^ (x >> 7)) + c,
 * 3 ops per step); 1: the same in 64 bits (3 ops per step, each a 64-bit operation); 2: 32-bit
 * funnel shift by a data-dependent amount (and + shift, 2 ops per step); 3: binary64 multiply and
 * add without FMA (2 ops per step); 4: random 8-byte reads from a 2 GiB buffer (one DRAM sector
 * each; the buffer is allocated from the library's pool for the call). Synchronizes `stream`; takes
 * a few milliseconds. Errors: INVALID_ARG (NULL ops_per_s, kind outside 0..4), OOM, CUDA. */
leco_status leco_probe_throughput(int32_t kind, double* ops_per_s, leco_stream_t stream);

/* ------------------------------------------------------------------------------------------ */
/* Column metadata and lifetime */

/* Sizes and parameters of the column (host memory *out, filled at once, no CUDA call). total_bytes
 * / (n * value bytes) is the compression ratio the paper reports (§4.3.1). Errors: INVALID_ARG. */
leco_status leco_stats_get(const leco_column* col, leco_stats* out);

/* Copy the column's stored format (§3.3 storage format): its m records (32 bytes each), padded
 * residual words and, for variable columns, m+1 starts, to caller-owned host buffers of at least
 * 32 m, 8 * (padded words) and 8 (m+1) bytes (any may be NULL to skip); synchronous. Errors:
 * INVALID_ARG, CUDA. */
leco_status leco_column_export(const leco_column* col, void* host_records, void* host_words,
                               void* host_starts);

/* Serialize to a self-describing host blob: the §3.3 storage format (records, starts for variable
 * columns, words) behind this library's 64-byte header and CRC-32. host_buf == NULL: *bytes = the
 * size needed. cap too small: INVALID_ARG with *bytes set. Synchronous (waits for the column's
 * encode). */
leco_status leco_serialize(const leco_column* col, void* host_buf, uint64_t cap, uint64_t* bytes);

/* Rebuild a column from a blob written by leco_serialize (§3.3 storage format). Everything a kernel
 * indexes with is validated on the host before any device work: magic, version, sizes, CRC, record
 * widths and dense offsets, starts tiling [0, n), zero padding, polynomial blocks the decoder can
 * evaluate. The blob stays the caller's. Errors: CORRUPT, INVALID_ARG, OOM, CUDA. */
leco_status leco_deserialize(const void* host_buf, uint64_t bytes, leco_stream_t stream,
                             leco_column** out);

/* Release a column: waits for the device to finish, then frees. NULL is ignored. Library
 * lifetime; the paper has no counterpart. */
void leco_column_free(leco_column* col);

/* Release a column in stream order: the memory is returned after the work already enqueued on
 * `stream` completes; the caller guarantees that no other stream still uses the column. Library
 * lifetime; the paper has no counterpart. */
void leco_column_free_async(leco_column* col, leco_stream_t stream);

/* Device memory: the library allocates from its own stream-ordered pool on each device, which keeps
 * freed memory cached for reuse. This call returns the cached memory of the current device's pool to
 * the driver (memory still owned by live columns stays). Synchronizes the device. Errors: CUDA.
 * A systems facility; the paper has no counterpart. */
leco_status leco_trim_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* LECO_H */
