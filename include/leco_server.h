/*
 * leco_server.h — request-serving loop of the GB300 LeCo library (libleco.so).
 *
 * The paper answers point lookups and range decompressions on one CPU thread (§3.3, §4.3); it has
 * no serving layer. This one keeps compressed columns resident on the device, admits columns
 * against a device-memory budget, and batches concurrent requests: a batcher thread turns the
 * queued requests into one batch whenever one of `max_inflight` slots is free (so requests that
 * arrive while others are on the GPU join the next batch), and each batch is one host-to-device
 * copy, one multi-column lookup kernel, one multi-column range-decode launch and one
 * device-to-host copy on the slot's own stream. A completer thread finishes requests in batch
 * order and stamps their latency. Each request's result is identical whether it runs alone or in a
 * batch (the same kernels compute every value independently).
 */
#ifndef LECO_SERVER_H
#define LECO_SERVER_H

#include "leco.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct leco_server leco_server;

typedef struct {
  uint64_t budget_bytes;        /* resident columns + every slot's device buffers must fit */
  uint32_t max_inflight;        /* batches on the GPU at once (slots), 1..16; 0 = 4 */
  uint32_t max_batch_requests;  /* requests per batch; 1 = one launch per request; 0 = 4096 */
  uint64_t max_batch_lookups;   /* lookup indices per batch (and per request); 0 = 1 << 20 */
  uint64_t max_batch_values;    /* range positions per batch (and per request); 0 = 1 << 25 */
  uint32_t max_columns;         /* column ids 0 .. max_columns-1; 0 = 4096 */
  uint32_t mock;                /* 1: host-only executor for tests (no GPU; see below) */
  uint32_t mock_batch_us;       /* mock: simulated time per batch */
} leco_server_config;

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t lookups, range_values; /* work completed */
  uint64_t batches, launches;     /* batches run, kernel launches issued */
  uint64_t max_batch_size;        /* most requests seen in one batch */
  double p50_us, p99_us, mean_us, max_us; /* submit -> completion latency */
  double elapsed_s;               /* since creation or the last reset */
  uint64_t resident_bytes;        /* device bytes of admitted columns */
  uint64_t reserved_bytes;        /* device bytes of the slots' buffers */
  uint32_t columns;               /* admitted columns */
} leco_server_stats;

/* Create a server on the current device (the serving layer; the paper has no counterpart). Errors:
 * INVALID_ARG, OOM, BUDGET (the slots alone do not fit in budget_bytes), CUDA. */
leco_status leco_server_create(const leco_server_config* cfg, leco_server** out);

/* Admit a column: on success the server owns it (it frees it on evict/destroy) and *col_id names
 * it in requests. BUDGET when resident + reserved + the column's device bytes > budget (the
 * caller keeps the column then). Serving layer; the paper has no counterpart. */
leco_status leco_server_admit(leco_server* s, leco_column* col, uint32_t* col_id);

/* Mock executor only: admit a column of n values of `dtype` occupying `bytes` (no device data).
 * Serving layer; the paper has no counterpart. */
leco_status leco_server_admit_mock(leco_server* s, uint64_t n, leco_dtype dtype, uint64_t bytes,
                                   uint32_t* col_id);

/* Remove a column once its pending requests are done, and free it.
 * Serving layer; the paper has no counterpart. */
leco_status leco_server_evict(leco_server* s, uint32_t col_id);

/* Queue k point lookups (§3.3 random access, served) of column col_id: host_idx is copied at
 * submit; host_out (k values of the column's width, host memory) is written before the request
 * completes and must stay valid until then. INDEX_RANGE when an index >= n, INVALID_ARG for an
 * unknown column or k over the batch limit. *req_id names the request for leco_server_wait. */
leco_status leco_server_submit_lookup(leco_server* s, uint32_t col_id, const uint64_t* host_idx,
                                      uint64_t k, void* host_out, uint64_t* req_id);

/* Queue the decode of positions [begin, begin + count) of column col_id (§3.3 range decompression,
 * served) into host_out (count values of the column's width, host memory, valid until the request
 * completes). INDEX_RANGE when begin + count > n, INVALID_ARG for an unknown column, count = 0 or
 * count over the batch limit. */
leco_status leco_server_submit_range(leco_server* s, uint32_t col_id, uint64_t begin, uint64_t count,
                                     void* host_out, uint64_t* req_id);

/* Wait up to timeout_ms for request req_id; on completion *result is its status and the request is
 * forgotten. TIMEOUT if still pending, INVALID_ARG for an unknown id.
 * Serving layer; the paper has no counterpart. */
leco_status leco_server_wait(leco_server* s, uint64_t req_id, uint32_t timeout_ms, leco_status* result);

/* Drive the server with a Poisson stream of requests for `seconds` at `rate` requests/s (seeded):
 * each request picks a column uniformly among `ncols` ids, then with probability lookup_frac is a
 * lookup of log-uniform 1..max_lookup uniform indices, else a range decode of log-uniform
 * min_range..max_range positions at a uniform start (clipped to the column). Output buffers are
 * the driver's own. Returns when every submitted request completed; *submitted = requests sent.
 * Serving layer; the paper has no counterpart. */
leco_status leco_server_drive_poisson(leco_server* s, const uint32_t* col_ids, uint32_t ncols, double rate,
                                      double seconds, uint64_t seed, double lookup_frac, uint64_t max_lookup,
                                      uint64_t min_range, uint64_t max_range, uint64_t* submitted);

/* Counters and latency percentiles since creation or the last reset (*out: host memory); reset
 * clears them and restarts the clock. Errors: INVALID_ARG. Serving layer; the paper has no
 * counterpart. */
leco_status leco_server_stats_get(leco_server* s, leco_server_stats* out);
leco_status leco_server_reset_stats(leco_server* s);

/* Finish queued requests, stop the threads, free the admitted columns and the slots.
 * Serving layer; the paper has no counterpart. */
void leco_server_destroy(leco_server* s);

#ifdef __cplusplus
}
#endif

#endif /* LECO_SERVER_H */
