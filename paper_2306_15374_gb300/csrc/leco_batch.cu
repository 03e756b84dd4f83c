// Batched decode plans and the scan autotuner (declared in include/leco_batch.h).
#include <string.h>

#include <vector>

#include "column.cuh"
#include "leco_batch.h"

using namespace leco;

namespace leco {
int tune_table_save(const char* path);
int tune_table_load(const char* path);
}  // namespace leco

struct leco_batch_plan {
  ColumnView* d_cols = nullptr;
  BatchItem* d_items = nullptr;
  uint32_t* d_status = nullptr;
  uint64_t nitems = 0;
  uint32_t stage_bytes = 64;
  ScanConfig cfg{4, 8};
  bool poly = false;  // some column has polynomial partitions
  int device = 0;
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void plan_release(leco_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->capture) cudaStreamDestroy(p->capture);
  if (p->d_cols) cudaFree(p->d_cols);
  if (p->d_items) cudaFree(p->d_items);
  if (p->d_status) cudaFree(p->d_status);
  delete p;
}

}  // namespace

extern "C" {

leco_status leco_tune_scan(const leco_column* col, uint32_t op, uint64_t lo, uint64_t hi,
                           leco_stream_t stream, leco_scan_config* best) {
  if (!col || !best || op > 1) return LECO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const ColumnView v = view_of(col);
  const uint64_t vb = col->dtype == LECO_U32 ? 4 : 8;
  void* buf = nullptr;
  cudaError_t e = dev_alloc(&buf, op == 0 ? (col->n ? col->n * vb : 8) : sizeof(leco_sum_result), st);
  if (e != cudaSuccess) return from_cuda(e);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const uint32_t stages[] = {2, 3, 4, 6, 8};
  const uint32_t warps[] = {4, 8};
  ScanConfig chosen{4, 8};
  float best_ms = -1.0f;
  for (uint32_t cw : warps) {
    for (uint32_t ns : stages) {
      const ScanConfig cfg{ns, cw};
      auto run = [&]() {
        return op == 0 ? launch_decode_cfg(v, 0, col->n, buf, cfg, st)
                       : launch_filter_sum_cfg(v, lo, hi, 0, (leco_sum_result*)buf, cfg, st);
      };
      if (run() != cudaSuccess) {  // e.g. too much shared memory for this column: skip
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(a, st);
      bool ok = true;
      for (int r = 0; r < 3 && ok; r++) ok = run() == cudaSuccess;
      cudaEventRecord(b, st);
      if (!ok || cudaEventSynchronize(b) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      ms /= 3.0f;
      if (best_ms < 0 || ms < best_ms) {
        best_ms = ms;
        chosen = cfg;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(buf, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  if (best_ms < 0) return LECO_ERR_CUDA;
  scan_config_store((int)op, col->dtype, col->stage_bytes, chosen);
  best->stages = chosen.stages;
  best->consumer_warps = chosen.consumer_warps;
  best->ms = best_ms;
  return LECO_OK;
}

leco_status leco_tune_save(const char* path) {
  if (!path) return LECO_ERR_INVALID_ARG;
  return tune_table_save(path) == 0 ? LECO_OK : LECO_ERR_INVALID_ARG;
}

leco_status leco_tune_load(const char* path) {
  if (!path) return LECO_ERR_INVALID_ARG;
  return tune_table_load(path) >= 0 ? LECO_OK : LECO_ERR_INVALID_ARG;
}

leco_status leco_batch_plan_create(const leco_column* const* cols, void* const* d_outs, uint32_t ncols,
                                   leco_batch_plan** out) {
  if (!out || (ncols && (!cols || !d_outs))) return LECO_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LECO_ERR_CUDA;
  std::vector<ColumnView> views(ncols);
  std::vector<BatchItem> items;
  uint32_t stage_bytes = 64;
  int dtype = LECO_U32;
  bool any_poly = false;
  for (uint32_t c = 0; c < ncols; c++) {
    const leco_column* col = cols[c];
    if (!col || col->device != dev || (col->n && !d_outs[c])) return LECO_ERR_INVALID_ARG;
    views[c] = view_of(col);
    any_poly = any_poly || col->poly != nullptr;
    stage_bytes = col->stage_bytes > stage_bytes ? col->stage_bytes : stage_bytes;
    if (col->dtype == LECO_U64) dtype = LECO_U64;
    const uint64_t vb = col->dtype == LECO_U32 ? 4 : 8;
    const uint64_t nt = scan_tiles(col->n);
    for (uint64_t t = 0; t < nt; t++) {
      BatchItem it;
      it.col = c;
      it.pad = 0;
      it.tile = t;
      it.begin = t * kScanTile;
      it.end = it.begin + kScanTile < col->n ? it.begin + kScanTile : col->n;
      it.out = static_cast<char*>(d_outs[c]) + it.begin * vb;
      items.push_back(it);
    }
  }
  leco_batch_plan* p = new (std::nothrow) leco_batch_plan();
  if (!p) return LECO_ERR_OOM;
  p->device = dev;
  p->nitems = items.size();
  p->stage_bytes = stage_bytes;
  p->poly = any_poly;
  p->cfg = scan_config_lookup(0, dtype, stage_bytes);
  cudaError_t e = cudaMalloc((void**)&p->d_cols, sizeof(ColumnView) * (ncols ? ncols : 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_items, sizeof(BatchItem) * (items.empty() ? 1 : items.size()));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_status, 256);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, 256);
  if (e == cudaSuccess && ncols)
    e = cudaMemcpy(p->d_cols, views.data(), sizeof(ColumnView) * ncols, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(p->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  // the memset and the copies from pageable memory ran on the legacy stream, and a copy may return
  // before its DMA lands: wait for them, so a run on any stream (non-blocking ones included) finds
  // the tables in place
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  if (e != cudaSuccess) {
    plan_release(p);
    return from_cuda(e);
  }
  *out = p;
  return LECO_OK;
}

leco_status leco_batch_plan_run(leco_batch_plan* plan, leco_stream_t stream) {
  if (!plan) return LECO_ERR_INVALID_ARG;
  return from_cuda(launch_batch_decode(plan->d_cols, plan->d_items, plan->nitems, plan->stage_bytes, plan->cfg,
                                       plan->poly, plan->d_status, (cudaStream_t)stream));
}

leco_status leco_batch_plan_run_graph(leco_batch_plan* plan, leco_stream_t stream) {
  if (!plan) return LECO_ERR_INVALID_ARG;
  if (!plan->exec) {
    cudaError_t e = plan->capture ? cudaSuccess : cudaStreamCreateWithFlags(&plan->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(plan->capture, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t le = launch_batch_decode(plan->d_cols, plan->d_items, plan->nitems, plan->stage_bytes,
                                                 plan->cfg, plan->poly, plan->d_status, plan->capture);
      e = cudaStreamEndCapture(plan->capture, &plan->graph);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&plan->exec, plan->graph, 0);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return from_cuda(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
}

leco_status leco_batch_plan_tune(leco_batch_plan* plan, leco_stream_t stream, leco_scan_config* best) {
  if (!plan || !best) return LECO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return LECO_ERR_CUDA;
  const uint32_t stages[] = {2, 3, 4, 6, 8};
  const uint32_t warps[] = {4, 8};
  ScanConfig chosen = plan->cfg;
  float best_ms = -1.0f;
  for (uint32_t cw : warps) {
    for (uint32_t ns : stages) {
      const ScanConfig cfg{ns, cw};
      auto run = [&]() {
        return launch_batch_decode(plan->d_cols, plan->d_items, plan->nitems, plan->stage_bytes, cfg,
                                   plan->poly, plan->d_status, st);
      };
      if (run() != cudaSuccess) {  // e.g. too much shared memory for the plan's widest tile: skip
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(a, st);
      const bool ok = run() == cudaSuccess && run() == cudaSuccess;
      cudaEventRecord(b, st);
      if (!ok || cudaEventSynchronize(b) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      ms /= 2.0f;
      if (best_ms < 0 || ms < best_ms) {
        best_ms = ms;
        chosen = cfg;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cudaStreamSynchronize(st) != cudaSuccess || best_ms < 0) return LECO_ERR_CUDA;
  if (chosen.stages != plan->cfg.stages || chosen.consumer_warps != plan->cfg.consumer_warps) {
    plan->cfg = chosen;
    if (plan->exec) {  // the captured graph holds the old launch shape: capture again on next use
      cudaGraphExecDestroy(plan->exec);
      plan->exec = nullptr;
    }
    if (plan->graph) {
      cudaGraphDestroy(plan->graph);
      plan->graph = nullptr;
    }
  }
  best->stages = chosen.stages;
  best->consumer_warps = chosen.consumer_warps;
  best->ms = best_ms;
  return LECO_OK;
}

leco_status leco_batch_plan_sync(leco_batch_plan* plan, leco_stream_t stream) {
  if (!plan) return LECO_ERR_INVALID_ARG;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LECO_ERR_CUDA;
  uint32_t flags = 0;
  if (cudaMemcpy(&flags, plan->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LECO_ERR_CUDA;
  // cleared in stream order and waited for, so a later run on any stream cannot have its flag erased
  if (flags && (cudaMemsetAsync(plan->d_status, 0, 4, (cudaStream_t)stream) != cudaSuccess ||
                cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess))
    return LECO_ERR_CUDA;
  if (flags & kStatTimeout) return LECO_ERR_TIMEOUT;
  if (flags & kStatCorrupt) return LECO_ERR_CORRUPT;
  if (flags & kStatIndexRange) return LECO_ERR_INDEX_RANGE;
  return LECO_OK;
}

uint64_t leco_batch_plan_jobs(const leco_batch_plan* plan) { return plan ? plan->nitems : 0; }

void leco_batch_plan_free(leco_batch_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  plan_release(plan);
}

leco_status leco_batch_decode(const leco_column* const* cols, void* const* d_outs, uint32_t ncols,
                              leco_stream_t stream) {
  leco_batch_plan* p = nullptr;
  leco_status s = leco_batch_plan_create(cols, d_outs, ncols, &p);
  if (s != LECO_OK) return s;
  s = leco_batch_plan_run(p, stream);
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  plan_release(p);
  if (s == LECO_OK && e != cudaSuccess) s = LECO_ERR_CUDA;
  return s;
}

}  // extern "C"

// ------------------------------------------------------------------------------ batched encode

namespace {

bool encode_args_ok(const void* const* d_vals, const uint64_t* n, const leco_model* models, const uint32_t* L,
                    uint32_t ncols, leco_dtype dtype) {
  if ((ncols && (!d_vals || !n || !models || !L)) || (dtype != LECO_U32 && dtype != LECO_U64)) return false;
  for (uint32_t c = 0; c < ncols; c++)
    if ((n[c] && !d_vals[c]) || L[c] < 1 || L[c] > kMaxPartLen ||
        (models[c] != LECO_MODEL_CONSTANT && models[c] != LECO_MODEL_LINEAR && models[c] != LECO_MODEL_POLY))
      return false;
  return true;
}

// Host tables of a batched encode (columns, first partition / scan tile of each column, pack items)
// and the layout of its device blocks:
//   meta:    records | decode table | tile descriptors | status words | polynomial table
//   scratch: lenbits | scan scratch | col_bits | max_b | polynomial blocks | part_col
struct EncBatch {
  uint32_t ncols = 0;
  int dtype = LECO_U64;
  bool any_poly = false;
  std::vector<EncCol> ec;
  std::vector<uint64_t> part_base, tile_base;
  std::vector<PackItem> items;
  uint64_t P = 0, T = 0;
  uint64_t rec_b = 0, tiles_b = 0, stat_b = 0, poly_b = 0, pc_words = 0, pcol_words = 0, scr_words = 0;

  EncBatch(const void* const* d_vals, const uint64_t* n, const leco_model* models, const uint32_t* L, uint32_t k,
           leco_dtype dt, EncodeConfig cfg)
      : ncols(k), dtype(dt), ec(k), part_base(k + 1), tile_base(k + 1) {
    for (uint32_t c = 0; c < ncols; c++) any_poly = any_poly || models[c] == LECO_MODEL_POLY;
    part_base[0] = tile_base[0] = 0;
    for (uint32_t c = 0; c < ncols; c++) {
      ec[c] = EncCol{d_vals[c], n[c], L[c], (int32_t)models[c]};
      part_base[c + 1] = part_base[c] + (n[c] + L[c] - 1) / L[c];
      tile_base[c + 1] = tile_base[c] + scan_tiles(n[c]);
    }
    P = part_base[ncols];
    T = tile_base[ncols];
    // pack items: runs of consecutive partitions of one column that fit one staged copy
    items.reserve(P / 4 + ncols);
    const uint64_t item_vals = cfg.item_values >= 1 && cfg.item_values <= pack_item_values() ? cfg.item_values
                                                                                             : pack_item_values();
    for (uint32_t c = 0; c < ncols; c++) {
      const uint64_t mc = part_base[c + 1] - part_base[c];
      const uint64_t g = models[c] == LECO_MODEL_POLY ? 1 : (L[c] >= item_vals ? 1 : item_vals / L[c]);
      for (uint64_t q = 0; q < mc; q += g)
        items.push_back(PackItem{part_base[c] + q, c, (uint32_t)(mc - q < g ? mc - q : g)});
    }
    auto a256 = [](uint64_t x) { return (x + 255) & ~255ull; };
    rec_b = a256(32 * (P ? P : 1));
    tiles_b = a256(sizeof(TileDesc) * (T ? T : 1));
    stat_b = a256(4ull * ncols);
    poly_b = any_poly ? a256(sizeof(PolyAux) * (P ? P : 1)) : 0;
    pc_words = any_poly ? (sizeof(PolyCoef) / 8) * (P ? P : 1) : 0;
    pcol_words = (P + 1) / 2 + 1;  // part_col, 32 bits per partition
    scr_words = P + offsets_multi_scratch_elems(P) + 2 * (uint64_t)ncols + 8 + pc_words + pcol_words;
  }
  uint64_t meta_bytes() const { return 2 * rec_b + tiles_b + stat_b + poly_b; }
};

// device pointers into the blocks of an EncBatch
struct EncPtrs {
  Record* rec;
  Aux* aux;
  TileDesc* tiles;
  uint32_t* status;
  PolyAux* poly;
  uint64_t *lenbits, *offs, *colbits;
  uint32_t* maxb;
  PolyCoef* pcoef;
  uint32_t* part_col;
};

EncPtrs enc_ptrs(const EncBatch& B, char* meta, uint64_t* scr) {
  EncPtrs p;
  p.rec = reinterpret_cast<Record*>(meta);
  p.aux = reinterpret_cast<Aux*>(meta + B.rec_b);
  p.tiles = reinterpret_cast<TileDesc*>(meta + 2 * B.rec_b);
  p.status = reinterpret_cast<uint32_t*>(meta + 2 * B.rec_b + B.tiles_b);
  p.poly = B.any_poly ? reinterpret_cast<PolyAux*>(meta + 2 * B.rec_b + B.tiles_b + B.stat_b) : nullptr;
  p.lenbits = scr;
  p.offs = scr + B.P;
  p.colbits = p.offs + offsets_multi_scratch_elems(B.P);
  p.maxb = reinterpret_cast<uint32_t*>(p.colbits + B.ncols);
  p.pcoef = B.any_poly ? reinterpret_cast<PolyCoef*>(scr + B.scr_words - B.pcol_words - B.pc_words) : nullptr;
  p.part_col = reinterpret_cast<uint32_t*>(scr + B.scr_words - B.pcol_words);
  return p;
}

// the device views the tile-descriptor pass reads (words and staging size are not read there)
std::vector<ColumnView> enc_views(const EncBatch& B, const EncPtrs& p, const uint64_t* n, const uint32_t* L) {
  std::vector<ColumnView> views(B.ncols);
  for (uint32_t c = 0; c < B.ncols; c++) {
    ColumnView& v = views[c];
    v.n = n[c];
    v.m = B.part_base[c + 1] - B.part_base[c];
    v.dtype = B.dtype;
    v.L = L[c];
    v.rec = p.rec + B.part_base[c];
    v.aux = p.aux + B.part_base[c];
    v.words = nullptr;
    v.starts = nullptr;
    v.tiles = p.tiles + B.tile_base[c];
    v.poly = B.ec[c].model == LECO_MODEL_POLY ? p.poly + B.part_base[c] : nullptr;
    v.stage_bytes = 0;
    v.status = p.status + c;
  }
  return views;
}

// One column handle per column over the shared blocks meta (laid out as B) and words; the handles
// take the blocks (released with the last of them).
cudaError_t make_batch_columns(const EncBatch& B, const EncPtrs& p, uint64_t* words,
                               const std::vector<uint64_t>& word_base, const std::vector<uint64_t>& col_bits,
                               const std::vector<uint32_t>& max_b, const leco_model* models, const uint32_t* L,
                               int dev, cudaStream_t st, char* meta, leco_column** out) {
  leco_shared_blocks* sh = new (std::nothrow) leco_shared_blocks();
  if (!sh) return cudaErrorMemoryAllocation;
  sh->blocks[0] = meta;
  sh->blocks[1] = words;
  sh->refs.store((int)B.ncols);
  for (uint32_t c = 0; c < B.ncols; c++) {
    leco_column* col = new leco_column();
    const bool pc = models[c] == LECO_MODEL_POLY;
    col->n = B.ec[c].n;
    col->m = B.part_base[c + 1] - B.part_base[c];
    col->total_bits = col_bits[c];
    col->nwords = word_base[c + 1] - word_base[c];
    col->dtype = B.dtype;
    col->kind = LECO_PART_FIXED;
    col->model = models[c];
    col->L = L[c];
    col->device = dev;
    col->rec = p.rec + B.part_base[c];
    col->aux = p.aux + B.part_base[c];
    col->tiles = p.tiles + B.tile_base[c];
    col->poly = pc ? p.poly + B.part_base[c] : nullptr;
    col->status = p.status + c;
    col->max_b = max_b[c];
    col->stage_bytes = stage_word_bytes(max_b[c]) + (pc ? kPolyStageExtra : 0);
    col->words = words + word_base[c];
    col->meta_bytes = (pc ? 64 + sizeof(PolyAux) : 64) * col->m + sizeof(TileDesc) * scan_tiles(col->n);
    col->words_bytes = 8 * col->nwords;
    col->home = st;
    col->shared = sh;
    out[c] = col;
  }
  return cudaSuccess;
}

leco_status batch_encode_cfg(const void* const* d_vals, const uint64_t* n, const leco_model* models,
                             const uint32_t* L, uint32_t ncols, leco_dtype dtype, leco_stream_t stream,
                             leco_column** out, EncodeConfig cfg) {
  if (!out) return LECO_ERR_INVALID_ARG;
  for (uint32_t c = 0; c < ncols; c++) out[c] = nullptr;
  if (!encode_args_ok(d_vals, n, models, L, ncols, dtype)) return LECO_ERR_INVALID_ARG;
  if (ncols == 0) return LECO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  const EncBatch B(d_vals, n, models, L, ncols, dtype, cfg);
  const uint64_t P = B.P, T = B.T, nitems = B.items.size();
  char* meta = nullptr;
  uint64_t* scr = nullptr;
  EncCol* d_ec = nullptr;
  uint64_t* d_bases = nullptr;  // part_base | tile_base | word_base
  ColumnView* d_views = nullptr;
  PackItem* d_items = nullptr;
  uint64_t* words = nullptr;
  std::vector<uint64_t> col_bits(ncols), word_base(ncols + 1);
  std::vector<uint32_t> max_b(ncols);
  uint64_t W = 0;
  cudaError_t e = dev_alloc((void**)&meta, B.meta_bytes(), st);
  if (e == cudaSuccess) e = dev_alloc((void**)&scr, 8 * B.scr_words, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&d_ec, sizeof(EncCol) * ncols, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&d_bases, 8 * 3 * (uint64_t)(ncols + 1), st);
  if (e == cudaSuccess) e = dev_alloc((void**)&d_views, sizeof(ColumnView) * ncols, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&d_items, sizeof(PackItem) * (nitems ? nitems : 1), st);
  const EncPtrs p = enc_ptrs(B, meta, scr);
  uint64_t* d_part = d_bases;
  uint64_t* d_tile = d_bases + (ncols + 1);
  uint64_t* d_word = d_bases + 2 * (ncols + 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.status, 0, B.stat_b, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ec, B.ec.data(), sizeof(EncCol) * ncols, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_part, B.part_base.data(), 8 * (ncols + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tile, B.tile_base.data(), 8 * (ncols + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nitems)
    e = cudaMemcpyAsync(d_items, B.items.data(), sizeof(PackItem) * nitems, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_part_col(d_part, ncols, P, p.part_col, st);
  // fit every partition of every column, then column-relative offsets and per-column totals
  if (e == cudaSuccess)
    e = launch_fit_multi(d_ec, d_part, p.part_col, ncols, P, dtype, p.rec, p.lenbits, p.pcoef, p.maxb, p.status,
                         cfg.fit_ctas, st);
  if (e == cudaSuccess) e = launch_offsets_multi(p.rec, p.lenbits, d_part, p.part_col, ncols, P, p.offs, p.colbits, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(col_bits.data(), p.colbits, 8 * ncols, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(max_b.data(), p.maxb, 4 * ncols, cudaMemcpyDeviceToHost, st);
  uint32_t fit_flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&fit_flags, p.status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && (fit_flags & kStatTimeout)) e = cudaErrorTimeout;  // a staging copy never landed
  if (e == cudaSuccess) {
    word_base[0] = 0;
    for (uint32_t c = 0; c < ncols; c++) {
      if (col_bits[c] >= (1ull << 48)) e = cudaErrorInvalidValue;
      word_base[c + 1] = word_base[c] + stream_words(col_bits[c]);
    }
    W = word_base[ncols];
  }
  if (e == cudaSuccess) e = dev_alloc((void**)&words, 8 * W, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_word, word_base.data(), 8 * (ncols + 1), cudaMemcpyHostToDevice, st);
  const std::vector<ColumnView> views = enc_views(B, p, n, L);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_views, views.data(), sizeof(ColumnView) * ncols, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_aux_multi(p.rec, p.pcoef, d_ec, d_part, p.part_col, P, p.aux, p.poly, st);
  if (e == cudaSuccess) e = launch_tile_desc_multi(d_views, d_tile, ncols, T, B.any_poly, p.tiles, st);
  if (e == cudaSuccess)
    e = launch_pack_multi(d_ec, d_part, p.part_col, d_word, p.colbits, d_items, nitems, ncols, P, W, dtype, p.rec,
                          p.aux, p.pcoef, p.poly, words, p.status, st);
  if (e == cudaSuccess) e = make_batch_columns(B, p, words, word_base, col_bits, max_b, models, L, dev, st, meta, out);
  cudaFreeAsync(scr, st);
  cudaFreeAsync(d_ec, st);
  cudaFreeAsync(d_bases, st);
  cudaFreeAsync(d_views, st);
  cudaFreeAsync(d_items, st);
  if (e != cudaSuccess) {
    if (meta) cudaFreeAsync(meta, st);
    if (words) cudaFreeAsync(words, st);
    return e == cudaErrorInvalidValue ? LECO_ERR_INVALID_ARG : from_cuda(e);
  }
  return LECO_OK;
}

}  // namespace

// A batched encode prepared once and replayed as one CUDA graph (leco_batch.h). The plan owns
// device copies of the host tables, the fit scratch, one meta block and a words block sized for the
// widest stream every column could have (64 bits per value plus the polynomial blocks), so that the
// packed streams' offsets are computed on the device and nothing waits on the host between the fit
// and the pack.
struct leco_batch_encode_plan {
  EncBatch* B = nullptr;
  std::vector<leco_model> models;
  std::vector<uint32_t> L;
  std::vector<uint64_t> n;
  int device = 0;
  EncodeConfig cfg{4096, 3};
  char* meta = nullptr;
  uint64_t* scr = nullptr;
  void* poly_scr = nullptr;
  EncCol* d_ec = nullptr;
  uint64_t* d_bases = nullptr;  // part_base | tile_base | word_base
  ColumnView* d_views = nullptr;
  PackItem* d_items = nullptr;
  uint64_t* words = nullptr;
  uint64_t words_cap = 0;  // 64-bit words reserved for the packed streams
  uint64_t runs = 0;       // graph launches so far
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void enc_plan_release(leco_batch_encode_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->capture) cudaStreamDestroy(p->capture);
  for (void* b : {(void*)p->meta, (void*)p->scr, p->poly_scr, (void*)p->d_ec, (void*)p->d_bases, (void*)p->d_views,
                  (void*)p->d_items, (void*)p->words})
    if (b) cudaFree(b);
  delete p->B;
  delete p;
}

// the graph's body: fit, offsets, word bases, decode table, tile descriptors, pack
cudaError_t enc_plan_launches(leco_batch_encode_plan* pl, cudaStream_t st) {
  const EncBatch& B = *pl->B;
  const EncPtrs p = enc_ptrs(B, pl->meta, pl->scr);
  uint64_t* d_part = pl->d_bases;
  uint64_t* d_tile = pl->d_bases + (B.ncols + 1);
  uint64_t* d_word = pl->d_bases + 2 * (B.ncols + 1);
  cudaError_t e = cudaMemsetAsync(p.status, 0, B.stat_b, st);
  if (e == cudaSuccess)
    e = launch_fit_multi(pl->d_ec, d_part, p.part_col, B.ncols, B.P, B.dtype, p.rec, p.lenbits, p.pcoef, p.maxb,
                         p.status, pl->cfg.fit_ctas, st, pl->poly_scr);
  if (e == cudaSuccess)
    e = launch_offsets_multi(p.rec, p.lenbits, d_part, p.part_col, B.ncols, B.P, p.offs, p.colbits, st);
  if (e == cudaSuccess) e = launch_word_bases(p.colbits, B.ncols, d_word, st);
  if (e == cudaSuccess) e = launch_aux_multi(p.rec, p.pcoef, pl->d_ec, d_part, p.part_col, B.P, p.aux, p.poly, st);
  if (e == cudaSuccess) e = launch_tile_desc_multi(pl->d_views, d_tile, B.ncols, B.T, B.any_poly, p.tiles, st);
  if (e == cudaSuccess)
    e = launch_pack_multi(pl->d_ec, d_part, p.part_col, d_word, p.colbits, pl->d_items, B.items.size(), B.ncols, B.P,
                          pl->words_cap, B.dtype, p.rec, p.aux, p.pcoef, p.poly, pl->words, p.status, st);
  return e;
}

}  // namespace

extern "C" leco_status leco_batch_encode(const void* const* d_vals, const uint64_t* n, const leco_model* models,
                                         const uint32_t* L, uint32_t ncols, leco_dtype dtype,
                                         leco_stream_t stream, leco_column** out) {
  return batch_encode_cfg(d_vals, n, models, L, ncols, dtype, stream, out, encode_config_lookup(dtype));
}

extern "C" leco_status leco_tune_batch_encode(const void* const* d_vals, const uint64_t* n, const leco_model* models,
                                              const uint32_t* L, uint32_t ncols, leco_dtype dtype,
                                              leco_stream_t stream, leco_encode_config* best) {
  if (!best || (dtype != LECO_U32 && dtype != LECO_U64)) return LECO_ERR_INVALID_ARG;
  if (ncols == 0) return LECO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<leco_column*> cols(ncols, nullptr);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return LECO_ERR_CUDA;
  }
  leco_status s = LECO_OK;
  EncodeConfig win{4096, 4};
  float win_ms = -1.f;
  const uint32_t items[3] = {1024, 2048, 4096}, ctas[3] = {2, 3, 4};
  for (int rep = 0; rep < 2 && s == LECO_OK; rep++) {  // the first pass warms pools and modules
    for (uint32_t iv : items)
      for (uint32_t fc : ctas) {
        if (s != LECO_OK) break;
        const EncodeConfig cfg{iv, fc};
        if (cudaEventRecord(e0, st) != cudaSuccess) s = LECO_ERR_CUDA;
        if (s == LECO_OK) s = batch_encode_cfg(d_vals, n, models, L, ncols, dtype, stream, cols.data(), cfg);
        if (s == LECO_OK && cudaEventRecord(e1, st) != cudaSuccess) s = LECO_ERR_CUDA;
        if (s == LECO_OK && cudaEventSynchronize(e1) != cudaSuccess) s = LECO_ERR_CUDA;
        float ms = 0.f;
        if (s == LECO_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) s = LECO_ERR_CUDA;
        for (leco_column*& c : cols) {
          leco_column_free_async(c, stream);
          c = nullptr;
        }
        if (s == LECO_OK && rep == 1 && (win_ms < 0.f || ms < win_ms)) {
          win_ms = ms;
          win = cfg;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != LECO_OK) return s;
  encode_config_store(dtype, win);
  best->item_values = win.item_values;
  best->fit_ctas = win.fit_ctas;
  best->ms = win_ms;
  return cudaStreamSynchronize(st) == cudaSuccess ? LECO_OK : LECO_ERR_CUDA;
}


extern "C" leco_status leco_batch_encode_plan_create(const void* const* d_vals, const uint64_t* n,
                                                     const leco_model* models, const uint32_t* L, uint32_t ncols,
                                                     leco_dtype dtype, leco_stream_t stream,
                                                     leco_batch_encode_plan** out) {
  if (!out) return LECO_ERR_INVALID_ARG;
  *out = nullptr;
  if (ncols == 0 || !encode_args_ok(d_vals, n, models, L, ncols, dtype)) return LECO_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LECO_ERR_CUDA;
  leco_batch_encode_plan* pl = new (std::nothrow) leco_batch_encode_plan();
  if (!pl) return LECO_ERR_OOM;
  pl->device = dev;
  pl->cfg = encode_config_lookup(dtype);
  pl->B = new (std::nothrow) EncBatch(d_vals, n, models, L, ncols, dtype, pl->cfg);
  if (!pl->B) {
    enc_plan_release(pl);
    return LECO_ERR_OOM;
  }
  const EncBatch& B = *pl->B;
  pl->models.assign(models, models + ncols);
  pl->L.assign(L, L + ncols);
  pl->n.assign(n, n + ncols);
  // the widest stream each column can have: 64 bits per value, plus a coefficient block per
  // partition long enough for a polynomial (at least kPolyMinLen values); below 2^41 values this
  // stays under the 2^48-bit offset field
  uint64_t cap = 0;
  for (uint32_t c = 0; c < ncols; c++) {
    if (n[c] >= (1ull << 41)) {
      enc_plan_release(pl);
      return LECO_ERR_INVALID_ARG;
    }
    const uint64_t m = B.part_base[c + 1] - B.part_base[c], mp = n[c] / kPolyMinLen;
    const uint64_t bits = 64 * n[c] + (models[c] == LECO_MODEL_POLY ? (uint64_t)kPolyBlockBits * (m < mp ? m : mp) : 0);
    cap += stream_words(bits);
  }
  pl->words_cap = cap;
  const uint64_t nitems = B.items.size();
  cudaError_t e = cudaMalloc((void**)&pl->meta, B.meta_bytes());
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->scr, 8 * B.scr_words);
  if (e == cudaSuccess && B.any_poly) e = cudaMalloc(&pl->poly_scr, poly_fit_scratch_bytes(B.P ? B.P : 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->d_ec, sizeof(EncCol) * ncols);
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->d_bases, 8 * 3 * (uint64_t)(ncols + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->d_views, sizeof(ColumnView) * ncols);
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->d_items, sizeof(PackItem) * (nitems ? nitems : 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&pl->words, 8 * cap);
  const EncPtrs p = enc_ptrs(B, pl->meta, pl->scr);
  const std::vector<ColumnView> views = enc_views(B, p, n, L);
  // the tables go in order on the caller's stream, ahead of the partition-column kernel that reads
  // them; the stream is synchronized below, before any graph run
  const cudaStream_t cst = (cudaStream_t)stream;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl->d_ec, B.ec.data(), sizeof(EncCol) * ncols, cudaMemcpyHostToDevice, cst);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl->d_bases, B.part_base.data(), 8 * (ncols + 1), cudaMemcpyHostToDevice, cst);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl->d_bases + (ncols + 1), B.tile_base.data(), 8 * (ncols + 1), cudaMemcpyHostToDevice, cst);
  if (e == cudaSuccess && nitems)
    e = cudaMemcpyAsync(pl->d_items, B.items.data(), sizeof(PackItem) * nitems, cudaMemcpyHostToDevice, cst);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(pl->d_views, views.data(), sizeof(ColumnView) * ncols, cudaMemcpyHostToDevice, cst);
  // the partition -> column table depends on the shapes only: filled once, outside the graph
  if (e == cudaSuccess) e = launch_part_col(pl->d_bases, ncols, B.P, p.part_col, cst);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cst);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(pl->capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t le = enc_plan_launches(pl, pl->capture);
    e = cudaStreamEndCapture(pl->capture, &pl->graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  if (e != cudaSuccess) {
    enc_plan_release(pl);
    return from_cuda(e);
  }
  *out = pl;
  return LECO_OK;
}

extern "C" leco_status leco_batch_encode_plan_run(leco_batch_encode_plan* plan, leco_stream_t stream) {
  if (!plan || !plan->exec) return LECO_ERR_INVALID_ARG;
  const cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
  if (e == cudaSuccess) plan->runs++;
  return from_cuda(e);
}

extern "C" leco_status leco_batch_encode_plan_columns(leco_batch_encode_plan* plan, leco_stream_t stream,
                                                      leco_column** out) {
  if (!plan || !out) return LECO_ERR_INVALID_ARG;
  const EncBatch& B = *plan->B;
  const uint32_t ncols = B.ncols;
  for (uint32_t c = 0; c < ncols; c++) out[c] = nullptr;
  if (plan->runs == 0) return LECO_ERR_INVALID_ARG;  // nothing encoded yet
  cudaStream_t st = (cudaStream_t)stream;
  const EncPtrs p = enc_ptrs(B, plan->meta, plan->scr);
  std::vector<uint64_t> col_bits(ncols), word_base(ncols + 1);
  std::vector<uint32_t> max_b(ncols), flags(ncols);
  cudaError_t e = cudaMemcpyAsync(col_bits.data(), p.colbits, 8 * ncols, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(max_b.data(), p.maxb, 4 * ncols, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags.data(), p.status, 4 * ncols, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  for (uint32_t c = 0; c < ncols; c++)
    if (flags[c] & kStatTimeout) return LECO_ERR_TIMEOUT;  // a staging copy never landed: streams incomplete
  word_base[0] = 0;
  for (uint32_t c = 0; c < ncols; c++) word_base[c + 1] = word_base[c] + stream_words(col_bits[c]);
  const uint64_t W = word_base[ncols];
  if (W > plan->words_cap) return LECO_ERR_CUDA;  // never: every stream is within its reserved width
  char* meta = nullptr;
  uint64_t* words = nullptr;
  e = dev_alloc((void**)&meta, B.meta_bytes(), st);
  if (e == cudaSuccess) e = dev_alloc((void**)&words, 8 * W, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(meta, plan->meta, B.meta_bytes(), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(words, plan->words, 8 * W, cudaMemcpyDeviceToDevice, st);
  int dev = plan->device;
  if (e == cudaSuccess)
    e = make_batch_columns(B, enc_ptrs(B, meta, plan->scr), words, word_base, col_bits, max_b, plan->models.data(),
                           plan->L.data(), dev, st, meta, out);
  if (e != cudaSuccess) {
    if (meta) cudaFreeAsync(meta, st);
    if (words) cudaFreeAsync(words, st);
    return from_cuda(e);
  }
  return LECO_OK;
}

extern "C" uint64_t leco_batch_encode_plan_reserved_bytes(const leco_batch_encode_plan* plan) {
  if (!plan) return 0;
  const EncBatch& B = *plan->B;
  const uint64_t nc = B.ncols;
  return B.meta_bytes() + 8 * B.scr_words + (B.any_poly ? poly_fit_scratch_bytes(B.P ? B.P : 1) : 0) +
         sizeof(EncCol) * nc + 8 * 3 * (nc + 1) + sizeof(ColumnView) * nc +
         sizeof(PackItem) * (B.items.empty() ? 1 : B.items.size()) + 8 * plan->words_cap;
}

extern "C" void leco_batch_encode_plan_free(leco_batch_encode_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  enc_plan_release(plan);
}
