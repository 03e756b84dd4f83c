// Request-serving loop (declared in include/leco_server.h): resident columns admitted against a
// device-memory budget, continuous batching of point lookups and range decodes into shared
// launches on up to max_inflight slots (stream + pinned/device buffers each), and latency stats.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "column.cuh"
#include "leco_server.h"

using namespace leco;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t id = 0;
  int type = 0;  // 0 lookup, 1 range
  uint32_t col = 0;
  int dtype = LECO_U64;
  std::vector<uint64_t> idx;
  uint64_t begin = 0, count = 0;
  void* out = nullptr;
  Clock::time_point t0;
  bool done = false;
  bool detached = false;  // issued by the load driver: nobody waits for it
  bool direct = false;    // out is pinned host memory: results are copied straight into it
  leco_status status = LECO_OK;
};

struct ColSlot {
  leco_column* col = nullptr;
  uint64_t n = 0;
  int dtype = LECO_U64;
  uint64_t bytes = 0;
  bool used = false, evicting = false;
  uint32_t pending = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t ldone = nullptr;  // the batch's lookup results are on the host
  cudaEvent_t done = nullptr;   // all of the batch's results are on the host
  bool lookups_done = false;    // lookup requests already completed
  Clock::time_point mock_done;  // mock executor: when the batch counts as finished
  uint64_t* h_idx = nullptr;
  uint32_t* h_col = nullptr;
  uint64_t* h_lout = nullptr;
  BatchItem* h_items = nullptr;
  unsigned char* h_rout = nullptr;
  uint64_t* d_idx = nullptr;
  uint32_t* d_col = nullptr;
  uint64_t* d_lout = nullptr;
  BatchItem* d_items = nullptr;
  unsigned char* d_rout = nullptr;
  std::vector<Req*> reqs;
  std::vector<uint64_t> off;  // lookups: first value; ranges: byte offset
  uint64_t nl = 0, nitems = 0, rbytes = 0, values = 0;
  uint32_t* d_stat = nullptr;  // device errors of the batch's range decode (kStat* flags)
  uint32_t* h_stat = nullptr;  // pinned copy, read when the batch is done
  cudaError_t err = cudaSuccess;
};

inline uint64_t vbytes(int dtype) { return dtype == LECO_U32 ? 4 : 8; }
inline uint64_t align16(uint64_t x) { return (x + 15) & ~15ull; }

}  // namespace

struct leco_server {
  leco_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> live;
  uint64_t next_id = 1;
  std::vector<ColSlot> cols;
  std::vector<ColumnView> h_views;
  ColumnView* d_views = nullptr;
  uint32_t stage_bytes = 64;
  bool poly = false;  // some admitted column has polynomial partitions
  uint64_t resident = 0, reserved = 0;
  uint64_t cap_items = 0;
  std::vector<Slot> slots;
  std::deque<int> free_slots, inflight;
  std::thread batcher, completer;
  bool stop = false, batcher_done = false;
  // statistics since creation / reset
  std::vector<double> lat_us;
  uint64_t submitted = 0, completed = 0, failed = 0, lookups = 0, range_values = 0, batches = 0, launches = 0,
           max_batch = 0, outstanding_detached = 0;
  Clock::time_point t_start;
};

namespace {

void slot_free(Slot& sl) {
  if (sl.stream) cudaStreamDestroy(sl.stream);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.ldone) cudaEventDestroy(sl.ldone);
  cudaFreeHost(sl.h_idx);
  cudaFreeHost(sl.h_col);
  cudaFreeHost(sl.h_lout);
  cudaFreeHost(sl.h_items);
  cudaFreeHost(sl.h_rout);
  cudaFree(sl.d_idx);
  cudaFree(sl.d_col);
  cudaFree(sl.d_lout);
  cudaFree(sl.d_items);
  cudaFree(sl.d_rout);
  cudaFree(sl.d_stat);
  cudaFreeHost(sl.h_stat);
}

uint64_t slot_device_bytes(const leco_server_config& c, uint64_t cap_items) {
  return c.max_batch_lookups * (8 + 4 + 8) + cap_items * sizeof(BatchItem) + 8 * c.max_batch_values +
         16 * (uint64_t)c.max_batch_requests;
}

cudaError_t slot_alloc(Slot& sl, const leco_server_config& c, uint64_t cap_items) {
  const uint64_t L = c.max_batch_lookups, rb = 8 * c.max_batch_values + 16 * (uint64_t)c.max_batch_requests;
  cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ldone, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_idx, 8 * L);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_col, 4 * L);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_lout, 8 * L);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_items, sizeof(BatchItem) * cap_items);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_rout, rb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_idx, 8 * L);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_col, 4 * L);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_lout, 8 * L);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_items, sizeof(BatchItem) * cap_items);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_rout, rb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_stat, 16);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_stat, 16);
  return e;
}

uint64_t tiles_of(uint64_t begin, uint64_t count) {
  return (begin + count - 1) / kScanTile - begin / kScanTile + 1;
}

// copy the batch's inputs to the slot and enqueue its GPU work (no lock held)
void gpu_run(leco_server* s, Slot& sl) {
  uint64_t nl = 0, ni = 0;
  for (size_t k = 0; k < sl.reqs.size(); k++) {
    Req* r = sl.reqs[k];
    if (r->type == 0) {
      for (uint64_t q = 0; q < r->idx.size(); q++) {
        sl.h_idx[nl + q] = r->idx[q];
        sl.h_col[nl + q] = r->col;
      }
      nl += r->idx.size();
    } else {
      const uint64_t vb = vbytes(r->dtype), end = r->begin + r->count;
      for (uint64_t t = r->begin / kScanTile; t * kScanTile < end; t++) {
        BatchItem& it = sl.h_items[ni++];
        it.col = r->col;
        it.pad = 0;
        it.tile = t;
        it.begin = std::max(t * kScanTile, r->begin);
        it.end = std::min((t + 1) * kScanTile, end);
        it.out = sl.d_rout + sl.off[k] + (it.begin - r->begin) * vb;
      }
    }
  }
  cudaError_t e = cudaSuccess;
  if (nl) {
    e = cudaMemcpyAsync(sl.d_idx, sl.h_idx, 8 * nl, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_col, sl.h_col, 4 * nl, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) e = launch_lookup_multi(s->d_views, sl.d_col, sl.d_idx, nl, sl.d_lout, sl.stream);
  }
  // results for pinned client buffers go straight there; the rest through the slot's staging
  bool staged_lookups = false, staged_ranges = false;
  for (size_t k = 0; k < sl.reqs.size() && e == cudaSuccess; k++) {
    const Req* r = sl.reqs[k];
    if (r->type == 0) {
      if (r->direct && r->dtype == LECO_U64)
        e = cudaMemcpyAsync(r->out, sl.d_lout + sl.off[k], 8 * r->idx.size(), cudaMemcpyDeviceToHost, sl.stream);
      else
        staged_lookups = true;
    } else if (!r->direct) {
      staged_ranges = true;
    }
  }
  if (nl && staged_lookups && e == cudaSuccess)
    e = cudaMemcpyAsync(sl.h_lout, sl.d_lout, 8 * nl, cudaMemcpyDeviceToHost, sl.stream);
  if (nl && e == cudaSuccess) e = cudaEventRecord(sl.ldone, sl.stream);  // lookups complete before ranges
  *sl.h_stat = 0;
  if (ni && e == cudaSuccess) {
    e = cudaMemsetAsync(sl.d_stat, 0, 4, sl.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sl.d_items, sl.h_items, sizeof(BatchItem) * ni, cudaMemcpyHostToDevice, sl.stream);
    uint32_t sb;
    bool poly;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      sb = s->stage_bytes;
      poly = s->poly;
    }
    if (e == cudaSuccess)
      e = launch_batch_decode(s->d_views, sl.d_items, ni, sb, scan_config_lookup(0, LECO_U64, sb), poly, sl.d_stat,
                              sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_stat, sl.d_stat, 4, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess && staged_ranges)
      e = cudaMemcpyAsync(sl.h_rout, sl.d_rout, sl.rbytes, cudaMemcpyDeviceToHost, sl.stream);
    for (size_t k = 0; k < sl.reqs.size() && e == cudaSuccess; k++) {
      const Req* r = sl.reqs[k];
      if (r->type == 1 && r->direct)
        e = cudaMemcpyAsync(r->out, sl.d_rout + sl.off[k], r->count * vbytes(r->dtype), cudaMemcpyDeviceToHost,
                            sl.stream);
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
  sl.nl = nl;
  sl.nitems = ni;
  sl.err = e;
}

void batcher_loop(leco_server* s) {
  if (!s->cfg.mock) cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return (s->stop && s->queue.empty()) || (!s->queue.empty() && !s->free_slots.empty()); });
    if (s->queue.empty()) break;  // stopping and drained
    const int si = s->free_slots.front();
    s->free_slots.pop_front();
    Slot& sl = s->slots[si];
    sl.reqs.clear();
    sl.off.clear();
    sl.nl = sl.nitems = sl.rbytes = sl.values = 0;
    sl.lookups_done = false;
    sl.err = cudaSuccess;
    uint64_t items = 0;
    // share the queue among the free slots: with idle slots, requests spread out (no waiting
    // behind each other's work); with one free slot, it takes everything queued (up to the caps)
    const uint64_t share = (s->queue.size() + s->free_slots.size()) / (s->free_slots.size() + 1);
    const uint64_t limit = std::min<uint64_t>(s->cfg.max_batch_requests, std::max<uint64_t>(1, share));
    while (!s->queue.empty() && sl.reqs.size() < limit) {
      Req* r = s->queue.front();
      uint64_t off;
      if (r->type == 0) {
        if (sl.nl + r->idx.size() > s->cfg.max_batch_lookups) break;
        off = sl.nl;
        sl.nl += r->idx.size();
      } else {
        const uint64_t t = tiles_of(r->begin, r->count);
        if (sl.values + r->count > s->cfg.max_batch_values || items + t > s->cap_items) break;
        off = sl.rbytes;
        sl.rbytes += align16(r->count * vbytes(r->dtype));
        sl.values += r->count;
        items += t;
      }
      s->queue.pop_front();
      sl.reqs.push_back(r);
      sl.off.push_back(off);
    }
    lk.unlock();
    if (s->cfg.mock)
      sl.mock_done = Clock::now() + std::chrono::microseconds(s->cfg.mock_batch_us);
    else
      gpu_run(s, sl);
    lk.lock();
    s->batches++;
    s->launches += s->cfg.mock ? 0 : (uint64_t)(sl.nl > 0) + (uint64_t)(sl.nitems > 0);
    s->max_batch = std::max<uint64_t>(s->max_batch, sl.reqs.size());
    s->inflight.push_back(si);
    s->cv.notify_all();
  }
  s->batcher_done = true;
  s->cv.notify_all();
}

// host-only executor: values are a fixed function of (column, position)
inline uint64_t mock_value(uint32_t col, uint64_t i) { return ((uint64_t)col << 40) ^ (i * 0x9E3779B97F4A7C15ull); }

// true once stage 0 (the slot's lookups) or stage 1 (all its work) has finished, or failed
bool slot_reached(leco_server* s, Slot& sl, int stage) {
  if (sl.err != cudaSuccess) return true;
  if (s->cfg.mock) return Clock::now() >= sl.mock_done;
  if (stage == 0 && sl.nl == 0) return true;
  const cudaError_t e = cudaEventQuery(stage == 0 ? sl.ldone : sl.done);
  if (e == cudaErrorNotReady) return false;
  if (e != cudaSuccess) sl.err = e;
  return true;
}

// Deliver the results of the slot's requests of one type (0 lookups, 1 ranges) whose GPU work has
// finished, then mark them done. A completed request's entry is cleared: its owner may free it.
void deliver(leco_server* s, Slot& sl, int type) {
  const cudaError_t e = sl.err;
  for (size_t k = 0; k < sl.reqs.size(); k++) {
    Req* r = sl.reqs[k];
    if (!r || r->type != type) continue;
    const uint64_t vb = vbytes(r->dtype);
    if (e != cudaSuccess) {
      r->status = e == cudaErrorLaunchTimeout ? LECO_ERR_TIMEOUT : LECO_ERR_CUDA;
      continue;
    }
    if (type == 1 && !s->cfg.mock && (*sl.h_stat & kStatTimeout)) {  // a bounded wait of the decode gave up
      r->status = LECO_ERR_TIMEOUT;
      continue;
    }
    if (r->direct && !s->cfg.mock && !(r->type == 0 && r->dtype == LECO_U32)) continue;  // already there
    if (r->type == 0) {
      const uint64_t o = sl.off[k];
      for (uint64_t q = 0; q < r->idx.size(); q++) {
        const uint64_t v = s->cfg.mock ? mock_value(r->col, r->idx[q]) : sl.h_lout[o + q];
        if (vb == 4)
          static_cast<uint32_t*>(r->out)[q] = (uint32_t)v;
        else
          static_cast<uint64_t*>(r->out)[q] = v;
      }
    } else if (s->cfg.mock) {
      for (uint64_t q = 0; q < r->count; q++) {
        const uint64_t v = mock_value(r->col, r->begin + q);
        if (vb == 4)
          static_cast<uint32_t*>(r->out)[q] = (uint32_t)v;
        else
          static_cast<uint64_t*>(r->out)[q] = v;
      }
    } else {
      memcpy(r->out, sl.h_rout + sl.off[k], r->count * vb);
    }
  }
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  for (Req*& r : sl.reqs) {
    if (!r || r->type != type) continue;
    r->done = true;
    const double us = std::chrono::duration<double, std::micro>(now - r->t0).count();
    s->lat_us.push_back(us);
    s->completed++;
    if (r->status != LECO_OK) s->failed++;
    if (r->type == 0)
      s->lookups += r->idx.size();
    else
      s->range_values += r->count;
    if (r->col < s->cols.size() && s->cols[r->col].pending) s->cols[r->col].pending--;
    if (r->detached) {
      s->outstanding_detached--;
      delete r;
    }
    r = nullptr;
  }
  s->cv.notify_all();
}

// Completes requests as their slots finish, in whatever order that happens: every in-flight slot
// is polled, its lookups complete when their results have landed (before the batch's range
// decodes), the rest when the batch is done, and the slot is then free for the batcher.
void completer_loop(leco_server* s) {
  if (!s->cfg.mock) cudaSetDevice(s->device);
  std::vector<int> flight;
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv.wait(lk, [&] { return !s->inflight.empty() || s->batcher_done; });
    if (s->inflight.empty()) break;  // the batcher has stopped and everything is delivered
    flight.assign(s->inflight.begin(), s->inflight.end());
    lk.unlock();
    bool progress = false;
    for (int si : flight) {
      Slot& sl = s->slots[si];
      if (!sl.lookups_done && slot_reached(s, sl, 0)) {
        deliver(s, sl, 0);
        sl.lookups_done = true;
        progress = true;
      }
      if (sl.lookups_done && slot_reached(s, sl, 1)) {
        deliver(s, sl, 1);
        std::lock_guard<std::mutex> lock(s->mu);
        sl.reqs.clear();
        s->inflight.erase(std::find(s->inflight.begin(), s->inflight.end(), si));
        s->free_slots.push_back(si);
        s->cv.notify_all();
        progress = true;
      }
    }
    if (!progress) std::this_thread::yield();
    lk.lock();
  }
}

leco_status submit(leco_server* s, Req* r, uint64_t* req_id) {
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return LECO_ERR_INVALID_ARG;
  if (r->col >= s->cols.size() || !s->cols[r->col].used || s->cols[r->col].evicting) return LECO_ERR_INVALID_ARG;
  const ColSlot& c = s->cols[r->col];
  r->dtype = c.dtype;
  if (r->type == 0) {
    if (r->idx.empty() || r->idx.size() > s->cfg.max_batch_lookups) return LECO_ERR_INVALID_ARG;
    for (uint64_t i : r->idx)
      if (i >= c.n) return LECO_ERR_INDEX_RANGE;
  } else {
    if (r->count == 0 || r->count > s->cfg.max_batch_values) return LECO_ERR_INVALID_ARG;
    if (r->begin > c.n || r->count > c.n - r->begin) return LECO_ERR_INDEX_RANGE;
    if (tiles_of(r->begin, r->count) > s->cap_items) return LECO_ERR_INVALID_ARG;
  }
  if (!s->cfg.mock) {
    cudaPointerAttributes attr;
    r->direct = cudaPointerGetAttributes(&attr, r->out) == cudaSuccess && attr.type == cudaMemoryTypeHost;
    cudaGetLastError();
  }
  r->id = s->next_id++;
  r->t0 = Clock::now();
  s->cols[r->col].pending++;
  s->submitted++;
  if (r->detached)
    s->outstanding_detached++;
  else
    s->live[r->id] = r;
  s->queue.push_back(r);
  if (req_id) *req_id = r->id;
  s->cv.notify_all();
  return LECO_OK;
}

leco_status admit_common(leco_server* s, leco_column* col, uint64_t n, int dtype, uint64_t bytes, uint32_t* col_id) {
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->resident + s->reserved + bytes > s->cfg.budget_bytes) return LECO_ERR_BUDGET;
  uint32_t id = 0;
  while (id < s->cols.size() && s->cols[id].used) id++;
  if (id >= s->cols.size()) return LECO_ERR_BUDGET;
  if (col) {
    s->h_views[id] = view_of(col);
    // a copy from pageable memory may return before its DMA lands, and the serving streams are
    // non-blocking: wait for the legacy stream, so the first batch that names this column finds it
    if (cudaMemcpy(s->d_views + id, &s->h_views[id], sizeof(ColumnView), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess)
      return LECO_ERR_CUDA;
    s->stage_bytes = std::max(s->stage_bytes, col->stage_bytes);
    s->poly = s->poly || col->poly != nullptr;
  }
  ColSlot& c = s->cols[id];
  c.col = col;
  c.n = n;
  c.dtype = dtype;
  c.bytes = bytes;
  c.used = true;
  c.evicting = false;
  c.pending = 0;
  s->resident += bytes;
  *col_id = id;
  return LECO_OK;
}

}  // namespace

extern "C" {

leco_status leco_server_create(const leco_server_config* cfg_in, leco_server** out) {
  if (!cfg_in || !out) return LECO_ERR_INVALID_ARG;
  *out = nullptr;
  leco_server_config cfg = *cfg_in;
  if (!cfg.max_inflight) cfg.max_inflight = 4;
  if (!cfg.max_batch_requests) cfg.max_batch_requests = 4096;
  if (!cfg.max_batch_lookups) cfg.max_batch_lookups = 1ull << 20;
  if (!cfg.max_batch_values) cfg.max_batch_values = 1ull << 25;
  if (!cfg.max_columns) cfg.max_columns = 4096;
  if (cfg.max_inflight > 16 || cfg.max_columns > (1u << 20)) return LECO_ERR_INVALID_ARG;
  leco_server* s = new (std::nothrow) leco_server();
  if (!s) return LECO_ERR_OOM;
  s->cfg = cfg;
  s->cols.resize(cfg.max_columns);
  s->cap_items = cfg.max_batch_values / kScanTile + 2ull * cfg.max_batch_requests + 16;
  s->slots.resize(cfg.max_inflight);
  s->t_start = Clock::now();
  if (!cfg.mock) {
    cudaGetDevice(&s->device);
    s->reserved = cfg.max_inflight * slot_device_bytes(cfg, s->cap_items) + sizeof(ColumnView) * cfg.max_columns;
    if (s->reserved > cfg.budget_bytes) {
      delete s;
      return LECO_ERR_BUDGET;
    }
    s->h_views.resize(cfg.max_columns);
    cudaError_t e = cudaMalloc((void**)&s->d_views, sizeof(ColumnView) * cfg.max_columns);
    for (uint32_t i = 0; i < cfg.max_inflight && e == cudaSuccess; i++) e = slot_alloc(s->slots[i], cfg, s->cap_items);
    if (e != cudaSuccess) {
      for (Slot& sl : s->slots) slot_free(sl);
      cudaFree(s->d_views);
      delete s;
      return from_cuda(e);
    }
  }
  for (uint32_t i = 0; i < cfg.max_inflight; i++) s->free_slots.push_back((int)i);
  s->batcher = std::thread(batcher_loop, s);
  s->completer = std::thread(completer_loop, s);
  *out = s;
  return LECO_OK;
}

leco_status leco_server_admit(leco_server* s, leco_column* col, uint32_t* col_id) {
  if (!s || !col || !col_id || s->cfg.mock) return LECO_ERR_INVALID_ARG;
  int dev = 0;
  cudaGetDevice(&dev);
  if (col->device != s->device) return LECO_ERR_INVALID_ARG;
  cudaStreamSynchronize(col->home);  // the column's encode is complete before batches read it
  return admit_common(s, col, col->n, col->dtype, col->meta_bytes + col->words_bytes, col_id);
}

leco_status leco_server_admit_mock(leco_server* s, uint64_t n, leco_dtype dtype, uint64_t bytes, uint32_t* col_id) {
  if (!s || !col_id || !s->cfg.mock || (dtype != LECO_U32 && dtype != LECO_U64)) return LECO_ERR_INVALID_ARG;
  return admit_common(s, nullptr, n, dtype, bytes, col_id);
}

leco_status leco_server_evict(leco_server* s, uint32_t col_id) {
  if (!s) return LECO_ERR_INVALID_ARG;
  leco_column* col = nullptr;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (col_id >= s->cols.size() || !s->cols[col_id].used || s->cols[col_id].evicting) return LECO_ERR_INVALID_ARG;
    s->cols[col_id].evicting = true;
    s->cv.wait(lk, [&] { return s->cols[col_id].pending == 0; });
    col = s->cols[col_id].col;
    s->resident -= s->cols[col_id].bytes;
    s->cols[col_id] = ColSlot();
  }
  if (col) leco_column_free(col);
  return LECO_OK;
}

leco_status leco_server_submit_lookup(leco_server* s, uint32_t col_id, const uint64_t* host_idx, uint64_t k,
                                      void* host_out, uint64_t* req_id) {
  if (!s || !host_idx || !host_out || !req_id) return LECO_ERR_INVALID_ARG;
  Req* r = new (std::nothrow) Req();
  if (!r) return LECO_ERR_OOM;
  r->type = 0;
  r->col = col_id;
  r->idx.assign(host_idx, host_idx + k);
  r->out = host_out;
  const leco_status st = submit(s, r, req_id);
  if (st != LECO_OK) delete r;
  return st;
}

leco_status leco_server_submit_range(leco_server* s, uint32_t col_id, uint64_t begin, uint64_t count,
                                     void* host_out, uint64_t* req_id) {
  if (!s || !host_out || !req_id) return LECO_ERR_INVALID_ARG;
  Req* r = new (std::nothrow) Req();
  if (!r) return LECO_ERR_OOM;
  r->type = 1;
  r->col = col_id;
  r->begin = begin;
  r->count = count;
  r->out = host_out;
  const leco_status st = submit(s, r, req_id);
  if (st != LECO_OK) delete r;
  return st;
}

leco_status leco_server_wait(leco_server* s, uint64_t req_id, uint32_t timeout_ms, leco_status* result) {
  if (!s) return LECO_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->live.find(req_id);
  if (it == s->live.end()) return LECO_ERR_INVALID_ARG;
  Req* r = it->second;
  if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) return LECO_ERR_TIMEOUT;
  if (result) *result = r->status;
  s->live.erase(it);
  delete r;
  return LECO_OK;
}

leco_status leco_server_drive_poisson(leco_server* s, const uint32_t* col_ids, uint32_t ncols, double rate,
                                      double seconds, uint64_t seed, double lookup_frac, uint64_t max_lookup,
                                      uint64_t min_range, uint64_t max_range, uint64_t* submitted) {
  if (!s || !col_ids || !ncols || !(rate > 0) || !(seconds >= 0) || max_lookup < 1 || min_range < 1 ||
      max_range < min_range)
    return LECO_ERR_INVALID_ARG;
  std::vector<uint64_t> ns(ncols);
  std::vector<int> dts(ncols);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    for (uint32_t c = 0; c < ncols; c++) {
      if (col_ids[c] >= s->cols.size() || !s->cols[col_ids[c]].used) return LECO_ERR_INVALID_ARG;
      ns[c] = s->cols[col_ids[c]].n;
      dts[c] = s->cols[col_ids[c]].dtype;
    }
  }
  // the driver's requests all write into one scratch buffer (their results are not kept), and at
  // most kWindow of them are outstanding: past that the driver waits, like a client with a
  // bounded number of connections
  constexpr uint64_t kWindow = 1u << 14;
  const uint64_t scratch_elems = std::max(max_lookup, max_range);
  std::vector<uint64_t> host_scratch;
  uint64_t* scratch = nullptr;
  if (s->cfg.mock || cudaMallocHost((void**)&scratch, 8 * scratch_elems) != cudaSuccess) {
    cudaGetLastError();
    host_scratch.resize(scratch_elems);
    scratch = host_scratch.data();
  }
  std::mt19937_64 rng(seed);
  std::exponential_distribution<double> gap(rate);
  std::uniform_real_distribution<double> u01(0.0, 1.0);
  const Clock::time_point t0 = Clock::now();
  double t = 0;
  uint64_t sent = 0;
  leco_status bad = LECO_OK;
  for (;;) {
    t += gap(rng);
    if (t > seconds) break;
    std::this_thread::sleep_until(t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(t)));
    const uint32_t c = (uint32_t)(u01(rng) * ncols) % ncols;
    const uint64_t n = ns[c];
    if (n == 0) continue;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->outstanding_detached < kWindow; });
    }
    Req* r = new Req();
    r->col = col_ids[c];
    r->detached = true;
    const uint64_t vb = vbytes(dts[c]);
    if (u01(rng) < lookup_frac) {
      const uint64_t k = std::max<uint64_t>(1, (uint64_t)std::exp(u01(rng) * std::log((double)max_lookup + 1)));
      r->type = 0;
      r->idx.resize(std::min<uint64_t>(k, max_lookup));
      for (auto& i : r->idx) i = (uint64_t)(u01(rng) * n) % n;
      r->out = scratch;
    } else {
      uint64_t cnt = (uint64_t)std::exp(std::log((double)min_range) +
                                        u01(rng) * (std::log((double)max_range) - std::log((double)min_range)));
      cnt = std::max<uint64_t>(1, std::min(cnt, n));
      r->type = 1;
      r->begin = (uint64_t)(u01(rng) * (double)(n - cnt + 1)) % (n - cnt + 1);
      r->count = cnt;
      r->out = scratch;
    }
    (void)vb;
    const leco_status st = submit(s, r, nullptr);
    if (st != LECO_OK) {
      delete r;
      bad = st;
      break;
    }
    sent++;
  }
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [&] { return s->outstanding_detached == 0; });
  }
  if (host_scratch.empty()) cudaFreeHost(scratch);
  if (submitted) *submitted = sent;
  return bad;
}

leco_status leco_server_stats_get(leco_server* s, leco_server_stats* out) {
  if (!s || !out) return LECO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->lookups = s->lookups;
  out->range_values = s->range_values;
  out->batches = s->batches;
  out->launches = s->launches;
  out->max_batch_size = s->max_batch;
  out->elapsed_s = std::chrono::duration<double>(Clock::now() - s->t_start).count();
  out->resident_bytes = s->resident;
  out->reserved_bytes = s->reserved;
  for (const ColSlot& c : s->cols) out->columns += c.used ? 1 : 0;
  if (!s->lat_us.empty()) {
    std::vector<double> v = s->lat_us;
    auto q = [&](double f) {
      const size_t k = std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + k, v.end());
      return v[k];
    };
    out->p50_us = q(0.50);
    out->p99_us = q(0.99);
    double sum = 0, mx = 0;
    for (double x : s->lat_us) {
      sum += x;
      mx = std::max(mx, x);
    }
    out->mean_us = sum / (double)s->lat_us.size();
    out->max_us = mx;
  }
  return LECO_OK;
}

leco_status leco_server_reset_stats(leco_server* s) {
  if (!s) return LECO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  s->lat_us.clear();
  s->submitted = s->completed = s->failed = s->lookups = s->range_values = s->batches = s->launches = s->max_batch = 0;
  s->t_start = Clock::now();
  return LECO_OK;
}

void leco_server_destroy(leco_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  s->batcher.join();
  s->completer.join();
  for (auto& kv : s->live) delete kv.second;
  if (!s->cfg.mock) {
    for (ColSlot& c : s->cols)
      if (c.used && c.col) leco_column_free(c.col);
    for (Slot& sl : s->slots) slot_free(sl);
    cudaFree(s->d_views);
  }
  delete s;
}

}  // extern "C"
