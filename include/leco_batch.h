/*
 * leco_batch.h — batched and tuned forms of the GB300 LeCo library (libleco.so).
 *
 * The paper decodes one column at a time on one CPU thread (§4.2); these calls are this library's
 * systems layer around the same per-value decode of §3.3: many columns of uneven lengths decoded
 * by one persistent kernel launch (optionally a CUDA graph) or encoded by one persistent fit and one
 * persistent pack launch (optionally a prepared plan replayed as one CUDA graph), and an autotuner
 * that picks the scan pipeline's and the encode's shape. Conventions (device pointers, streams,
 * ownership, errors) are those of leco.h.
 */
#ifndef LECO_BATCH_H
#define LECO_BATCH_H

#include "leco.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Shape of the scan pipeline: shared-memory stages in flight per CTA (2..8) and consumer warps
 * (4 or 8); ms is the measured time of the chosen configuration (leco_tune_scan only). */
typedef struct {
  uint32_t stages;
  uint32_t consumer_warps;
  double ms;
} leco_scan_config;

/* Time every candidate configuration of the scan on this column (op 0: leco_decode_all; op 1:
 * leco_filter_sum over [lo, hi] with flags 0), keep the fastest in the process-wide tuning table
 * (keyed by op, value width and the column's widest partition), and return it in *best. Later
 * decodes and filter-sums of columns in the same key use it; no result changes, only the speed.
 * Synchronizes `stream`; allocates a temporary decode output. Errors: INVALID_ARG, OOM, CUDA. An
 * autotuner of this library; the paper has no counterpart. */
leco_status leco_tune_scan(const leco_column* col, uint32_t op, uint64_t lo, uint64_t hi,
                           leco_stream_t stream, leco_scan_config* best);

/* Write / read the tuning table as JSON (host file path; host-only, no CUDA call). Save writes every
 * entry, one per line. Load merges the file's entries into the process-wide table, keeping those
 * that name a candidate the tuners can pick (scan: 2..8 stages, 4 or 8 consumer warps; batched
 * encode: 1024, 2048 or 4096 values per pack item, 2..4 fit CTAs per SM) and skipping the rest.
 * Errors: INVALID_ARG for a NULL path or a file that cannot be opened. The paper has no
 * counterpart. */
leco_status leco_tune_save(const char* path);
leco_status leco_tune_load(const char* path);

/* A prepared multi-column decode (the §3.3 Decoder over many columns; the batching is this library's
 * systems layer): every scan tile of every column becomes one job of a work table on the device,
 * so all columns decode in one persistent kernel launch. d_outs[c] receives
 * all values of cols[c] (n * value bytes, caller-owned, device). Columns may mix 32- and 64-bit
 * values and partition kinds; all must live on the current device. The plan owns its tables and
 * must be freed with leco_batch_plan_free; the columns must outlive it. */
typedef struct leco_batch_plan leco_batch_plan;

leco_status leco_batch_plan_create(const leco_column* const* cols, void* const* d_outs, uint32_t ncols,
                                   leco_batch_plan** out);

/* One kernel launch on `stream` decoding every column of the plan. Errors: INVALID_ARG (NULL
 * plan), CUDA; device-side errors surface at leco_batch_plan_sync.
 * Batching layer; the paper has no counterpart. */
leco_status leco_batch_plan_run(leco_batch_plan* plan, leco_stream_t stream);

/* The same launch as a CUDA graph: the first call captures it (on a private stream) and
 * instantiates the graph; every call launches the graph on `stream`. Errors as
 * leco_batch_plan_run. Batching layer; the paper has no counterpart. */
leco_status leco_batch_plan_run_graph(leco_batch_plan* plan, leco_stream_t stream);

/* Time the plan's launch under every candidate pipeline shape (the whole multi-column decode, on
 * `stream`, writing the plan's outputs) and keep the fastest for this plan's later runs; a graph
 * captured with another shape is captured again on its next run. The process-wide table of
 * leco_tune_scan is not changed. Synchronizes `stream`. Errors: INVALID_ARG, CUDA.
 * Batching layer; the paper has no counterpart. */
leco_status leco_batch_plan_tune(leco_batch_plan* plan, leco_stream_t stream, leco_scan_config* best);

/* Synchronize `stream`, then return the first device-side error the plan's runs recorded since the
 * last call (LECO_ERR_TIMEOUT when a bounded wait inside the decode gave up) and clear it, else
 * LECO_OK; a failed synchronization returns LECO_ERR_CUDA.
 * Batching layer; the paper has no counterpart. */
leco_status leco_batch_plan_sync(leco_batch_plan* plan, leco_stream_t stream);

/* Number of jobs (scan tiles) in the plan; 0 for NULL.
 * Batching layer; the paper has no counterpart. */
uint64_t leco_batch_plan_jobs(const leco_batch_plan* plan);

/* Waits for the device, then releases the plan's tables and graph. NULL is ignored.
 * Batching layer; the paper has no counterpart. */
void leco_batch_plan_free(leco_batch_plan* plan);

/* The §3.3 Decoder over many columns in one call: create + run + free (synchronizes `stream`
 * before freeing). Arguments and errors as leco_batch_plan_create and leco_batch_plan_run. */
leco_status leco_batch_decode(const leco_column* const* cols, void* const* d_outs, uint32_t ncols,
                              leco_stream_t stream);

/* Fixed-partition encode of ncols columns at once (§3.2.1 partitions, §3.1 fit, §3.3 packing):
 * column c has n[c] values of `dtype` at d_vals[c] (device), model models[c] (constant, linear or
 * polynomial, mixed freely) and partition size L[c] (1 .. 2^24). Every stage runs over all columns
 * in one launch (fit, offset scan, decode table, tile descriptors, pack; the polynomial columns' fit
 * adds its four phases over all their partitions), in the shape the tuning table holds for `dtype`
 * (leco_tune_batch_encode); one stream synchronization reads back the residual streams' sizes, which
 * the allocation of the packed streams needs. out[c] receives a column identical to
 * leco_encode(d_vals[c], n[c], dtype, fixed(L[c]), models[c]);
 * the columns share their device blocks, which are released when the last of them is freed.
 * Errors: INVALID_ARG, OOM, CUDA (then no column is returned). */
leco_status leco_batch_encode(const void* const* d_vals, const uint64_t* n, const leco_model* models,
                              const uint32_t* L, uint32_t ncols, leco_dtype dtype, leco_stream_t stream,
                              leco_column** out);

/* Shape of the batched encode (a systems knob; the paper has no counterpart): values per pack item
 * (1024, 2048 or 4096: a run of consecutive short partitions of one column that the packer stages
 * with one copy and packs in one CTA) and fit CTAs per SM (2, 3 or 4: fewer keep more of each
 * partition in L2 between the fit's two passes, more hide the exact solve's latency); ms is the
 * measured time of the chosen shape (leco_tune_batch_encode only). */
typedef struct {
  uint32_t item_values;
  uint32_t fit_ctas;
  double ms;
} leco_encode_config;

/* Time leco_batch_encode of these columns (arguments as there) under every candidate shape (twice;
 * the second pass counts), keep the fastest for later batched encodes of the same value width (the
 * process-wide tuning table, saved and loaded with the scan configurations), and return it in
 * *best. The encoded columns are freed; the result of every later encode is unchanged (byte for
 * byte), only its speed. Synchronizes `stream`. Errors: INVALID_ARG, OOM, CUDA. An autotuner of
 * this library; the paper has no counterpart. */
leco_status leco_tune_batch_encode(const void* const* d_vals, const uint64_t* n, const leco_model* models,
                                   const uint32_t* L, uint32_t ncols, leco_dtype dtype, leco_stream_t stream,
                                   leco_encode_config* best);

/* A prepared batched encode replayed as one CUDA graph (§3.2.1 partitions, §3.1 fit, §3.3 packing,
 * as leco_batch_encode; the batching itself is this library's systems layer). Creation does the
 * host work once: the columns' tables and pack items go to the device, the plan reserves its device
 * blocks (records, decode table, tile descriptors, fit scratch, and words for the widest stream each
 * column could have: 64 bits per value plus a polynomial coefficient block per partition that could
 * hold one), and the launches from the fit to the pack are captured in a CUDA graph in the encode
 * shape the tuning table holds for `dtype`. Each run is then one graph launch with no host round
 * trip: the streams' offsets are computed on the device, each column's stream placed right after the
 * previous one in the reserved words. Arguments as for leco_batch_encode, except that ncols must be
 * at least 1 and every n[c] below 2^41. The graph holds the pointers d_vals[c]: those buffers must
 * stay allocated while the plan lives, and each run encodes their contents at the time it runs.
 * Synchronizes `stream` once. Errors: INVALID_ARG, OOM (the reservation did not fit), CUDA. */
typedef struct leco_batch_encode_plan leco_batch_encode_plan;

leco_status leco_batch_encode_plan_create(const void* const* d_vals, const uint64_t* n, const leco_model* models,
                                          const uint32_t* L, uint32_t ncols, leco_dtype dtype, leco_stream_t stream,
                                          leco_batch_encode_plan** out);

/* One launch of the plan's graph on `stream`: every column is encoded (§3.1 fit, §3.3 packing)
 * into the plan's blocks, replacing the previous run's result. Runs that overlap on the device race
 * on those blocks. Errors: INVALID_ARG (NULL plan), CUDA; a bounded wait that gave up surfaces at
 * leco_batch_encode_plan_columns. */
leco_status leco_batch_encode_plan_run(leco_batch_encode_plan* plan, leco_stream_t stream);

/* Synchronize `stream` (the stream of the last run), then copy the last run's result out into
 * ncols new columns, out[c] identical to leco_batch_encode's out[c] for the same values: one block
 * of the records, decode table and tile descriptors and one of the packed streams at their exact
 * size, shared by the columns and released when the last of them is freed. The plan is unchanged
 * and may run again. Errors: INVALID_ARG (also before the plan's first run), OOM, TIMEOUT (a
 * bounded wait inside the run gave up; the streams are incomplete and no column is returned),
 * CUDA. Batching layer; the paper has no counterpart. */
leco_status leco_batch_encode_plan_columns(leco_batch_encode_plan* plan, leco_stream_t stream, leco_column** out);

/* Device bytes the plan holds (its tables, scratch and reserved words); 0 for NULL. The paper has no
 * counterpart. */
uint64_t leco_batch_encode_plan_reserved_bytes(const leco_batch_encode_plan* plan);

/* Waits for the device, then releases the plan's blocks and graph. NULL is ignored.
 * Batching layer; the paper has no counterpart. */
void leco_batch_encode_plan_free(leco_batch_encode_plan* plan);

#ifdef __cplusplus
}
#endif

#endif /* LECO_BATCH_H */
