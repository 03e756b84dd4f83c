// Internal layout of a leco_column (the opaque handle of include/leco.h), shared by the C-ABI
// modules of the library.
#pragma once

#include <atomic>

#include "leco_internal.cuh"

// Device blocks shared by the columns of one batched encode; freed when the last column goes.
struct leco_shared_blocks {
  std::atomic<int> refs{0};
  void* blocks[4] = {nullptr, nullptr, nullptr, nullptr};
};

struct leco_column {
  uint64_t n = 0;
  uint64_t m = 0;
  uint64_t nwords = 0;
  uint64_t total_bits = 0;
  int32_t dtype = LECO_U64;
  int32_t kind = LECO_PART_FIXED;
  int32_t model = LECO_MODEL_LINEAR;
  uint32_t L = 0;
  double tau = 0.0;
  int device = 0;
  leco::Record* rec = nullptr;
  leco::Aux* aux = nullptr;
  uint64_t* starts = nullptr;  // variable only
  leco::TileDesc* tiles = nullptr;   // scan tile descriptors
  leco::PolyAux* poly = nullptr;     // polynomial decode table (LECO_MODEL_POLY columns)
  uint32_t* status = nullptr;
  uint32_t max_b = 0;          // widest partition
  uint32_t stage_bytes = 0;    // shared-memory bytes per staged scan tile
  uint64_t* words = nullptr;
  void* meta_block = nullptr;
  uint64_t meta_bytes = 0;
  uint64_t words_bytes = 0;
  cudaStream_t home = nullptr;  // stream the column was created on
  leco_shared_blocks* shared = nullptr;  // batched encode: blocks shared with other columns
};

namespace leco {

inline leco_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return LECO_OK;
  if (e == cudaErrorMemoryAllocation) return LECO_ERR_OOM;
  if (e == cudaErrorTimeout) return LECO_ERR_TIMEOUT;  // a bounded device wait gave up (reported by the host)
  return LECO_ERR_CUDA;
}

inline ColumnView view_of(const leco_column* c) {
  ColumnView v;
  v.n = c->n;
  v.m = c->m;
  v.dtype = c->dtype;
  v.L = c->kind == LECO_PART_FIXED ? c->L : 0;
  v.rec = c->rec;
  v.aux = c->aux;
  v.words = c->words;
  v.starts = c->kind == LECO_PART_VAR ? c->starts : nullptr;
  v.tiles = c->tiles;
  v.poly = c->poly;
  v.stage_bytes = c->stage_bytes;
  v.status = c->status;
  return v;
}

}  // namespace leco
