// C ABI of the GB300 LeCo library (declared in include/leco.h): argument checking, column
// lifetime, the encode pipeline (partition -> fit -> offsets -> pack), the decode entry points
// and the self-describing blob (header + records + starts + words, CRC-32).
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "column.cuh"
#include "var_partition.cuh"

using namespace leco;

namespace {

// a named range on the profiler timeline for the duration of one C-ABI call (no cost without a tool)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxDevices] = {};

cudaMemPool_t pool_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

constexpr uint32_t kMagic = 0x4F43454Cu;  // "LECO"
constexpr uint32_t kVersion = 1;
constexpr uint64_t kHeaderBytes = 64;

inline uint64_t value_bytes(int dtype) { return dtype == LECO_U32 ? 4 : 8; }

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

// Allocate the metadata block (records, decode table, starts for variable columns, status).
leco_status alloc_meta(leco_column* c, cudaStream_t st) {
  const uint64_t rec_b = align256(32 * (c->m ? c->m : 1));
  const uint64_t starts_b = c->kind == LECO_PART_VAR ? align256(8 * (c->m + 1)) : 0;
  const uint64_t tiles_b = align256(sizeof(TileDesc) * (scan_tiles(c->n) + 1));
  const uint64_t poly_b = c->model == LECO_MODEL_POLY ? align256(sizeof(PolyAux) * (c->m ? c->m : 1)) : 0;
  c->meta_bytes = 2 * rec_b + starts_b + tiles_b + 256 + poly_b;
  void* p = nullptr;
  cudaError_t e = dev_alloc(&p, c->meta_bytes, st);
  if (e != cudaSuccess) return from_cuda(e);
  char* b = (char*)p;
  c->meta_block = p;
  c->rec = (Record*)b;
  c->aux = (Aux*)(b + rec_b);
  c->starts = starts_b ? (uint64_t*)(b + 2 * rec_b) : nullptr;
  c->tiles = (TileDesc*)(b + 2 * rec_b + starts_b);
  c->status = (uint32_t*)(b + 2 * rec_b + starts_b + tiles_b);
  c->poly = poly_b ? (PolyAux*)(b + 2 * rec_b + starts_b + tiles_b + 256) : nullptr;
  return from_cuda(cudaMemsetAsync(c->status, 0, 256, st));
}

void release(leco_column* c, cudaStream_t st) {
  if (!c) return;
  if (c->shared) {
    if (c->shared->refs.fetch_sub(1) == 1) {
      for (void* b : c->shared->blocks)
        if (b) cudaFreeAsync(b, st);
      delete c->shared;
    }
    delete c;
    return;
  }
  if (c->words) cudaFreeAsync(c->words, st);
  if (c->meta_block) cudaFreeAsync(c->meta_block, st);
  delete c;
}

// fit + offsets + pack of an already partitioned column (c->m, c->starts or c->L set). prefit: the
// records already hold every partition's fit (variable partitions fitted by the partitioner)
leco_status encode_partitions(leco_column* c, const void* d_values, cudaStream_t st, bool prefit = false) {
  const uint64_t m = c->m;
  const bool poly = c->model == LECO_MODEL_POLY;
  const uint64_t pc_elems = poly ? (sizeof(PolyCoef) / 8) * (m ? m : 1) : 0;
  const uint64_t scr_elems = m + offsets_scratch_elems(m) + 2 + pc_elems;
  uint64_t* scr = nullptr;
  cudaError_t e = dev_alloc((void**)&scr, scr_elems * 8, st);
  if (e != cudaSuccess) return from_cuda(e);
  uint64_t* lenbits = scr;
  uint64_t* off_scr = scr + m;
  uint64_t* d_total = scr + m + offsets_scratch_elems(m);  // [total bits, max width]
  uint32_t* d_maxb = reinterpret_cast<uint32_t*>(d_total + 1);
  PolyCoef* pcoef = poly ? reinterpret_cast<PolyCoef*>(d_total + 2) : nullptr;
  const uint64_t* starts = c->kind == LECO_PART_VAR ? c->starts : nullptr;
  uint64_t hres[2] = {0, 0};
  uint64_t& total = hres[0];
  uint32_t flags = 0;
  if (prefit)
    e = launch_lenbits(c->rec, starts, m, lenbits, d_maxb, st);
  else
    e = launch_fit(d_values, c->dtype, c->n, starts, c->L, m, c->model, c->rec, lenbits, pcoef, d_maxb, c->status,
                   st);
  if (e == cudaSuccess)
    e = launch_offsets(c->rec, lenbits, m, off_scr, offsets_scratch_elems(m), d_total, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hres, d_total, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, c->status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && (flags & kStatTimeout)) {
    cudaFreeAsync(scr, st);
    return LECO_ERR_TIMEOUT;  // a staging copy never landed: the fit is incomplete
  }
  if (e == cudaSuccess && total >= (1ull << 48)) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    c->total_bits = total;
    c->max_b = (uint32_t)hres[1];
    c->stage_bytes = stage_word_bytes(c->max_b) + (poly ? kPolyStageExtra : 0);
    c->nwords = stream_words(total);
    c->words_bytes = c->nwords * 8;
    e = dev_alloc((void**)&c->words, c->words_bytes, st);
  }
  if (e == cudaSuccess) e = launch_build_aux(c->rec, pcoef, m, c->n, c->aux, c->poly, c->status, st);
  if (e == cudaSuccess) e = launch_tile_desc(view_of(c), c->tiles, st);
  if (e == cudaSuccess) {
    if (c->kind == LECO_PART_VAR && !poly)
      e = launch_pack_var(d_values, c->dtype, c->rec, c->aux, m, c->n, total, c->words, c->nwords, c->status, st);
    else
      e = launch_pack(d_values, c->dtype, c->rec, c->aux, pcoef, c->poly, m, c->n, total, c->words, c->nwords,
                      c->status, st);
  }
  cudaFreeAsync(scr, st);
  if (e == cudaErrorInvalidValue) return LECO_ERR_INVALID_ARG;
  return from_cuda(e);
}

bool valid_dtype(int d) { return d == LECO_U32 || d == LECO_U64; }
bool valid_model(int m) { return m == LECO_MODEL_CONSTANT || m == LECO_MODEL_LINEAR || m == LECO_MODEL_POLY; }

// the model that sizes partitions for the variable partitioner and the size search: the polynomial
// model's choice is made per partition after partitioning, with the line's sizes before it
int sizing_model(int m) { return m == LECO_MODEL_POLY ? LECO_MODEL_LINEAR : m; }

// ---------------------------------------------------------------------------- CRC-32 (IEEE 802.3)

uint32_t crc_table[256];
std::once_flag crc_once;

void crc_init() {
  for (uint32_t i = 0; i < 256; i++) {
    uint32_t c = i;
    for (int k = 0; k < 8; k++) c = (c & 1) ? (0xEDB88320u ^ (c >> 1)) : (c >> 1);
    crc_table[i] = c;
  }
}

uint32_t crc32_update(uint32_t crc, const void* data, uint64_t len) {
  std::call_once(crc_once, crc_init);
  const uint8_t* p = (const uint8_t*)data;
  uint32_t c = ~crc;
  for (uint64_t i = 0; i < len; i++) c = crc_table[(c ^ p[i]) & 0xFF] ^ (c >> 8);
  return ~c;
}

struct BlobHeader {
  uint32_t magic;
  uint32_t version;
  uint64_t n;
  uint64_t m;
  uint64_t nwords;
  uint8_t dtype, kind, model, reserved0;
  uint32_t L;
  double tau;
  uint64_t total_bits;
  uint32_t crc;
  uint32_t reserved1;
};
static_assert(sizeof(BlobHeader) == kHeaderBytes, "blob header layout");

uint64_t blob_bytes(const leco_column* c) {
  return kHeaderBytes + 32 * c->m + (c->kind == LECO_PART_VAR ? 8 * (c->m + 1) : 0) + 8 * c->nwords;
}

// 64-bit field at bit pos of a stream held on the host (pos + 64 <= 64 * nwords)
uint64_t host_field64(const uint64_t* words, uint64_t pos) {
  const uint64_t w = pos >> 6;
  const uint32_t o = (uint32_t)(pos & 63);
  return o ? (words[w] >> o) | (words[w + 1] << (64 - o)) : words[w];
}

// a polynomial partition's block {T, K1, K2, K3, E} read from the stream at bit pos
PolyCoef host_poly_block(const uint64_t* words, uint64_t pos) {
  PolyCoef pc;
  pc.T = (int64_t)host_field64(words, pos);
  for (int j = 0; j < 3; j++) pc.K[j] = (int64_t)host_field64(words, pos + 64 * (uint64_t)(j + 1));
  pc.E = host_field64(words, pos + 256);
  return pc;
}

// a block the decoder can evaluate exactly: exponents 0..62 in the low three bytes, |K_j| <= 2^61,
// and each nonzero term K_j 2^(S - s_j) p_j below 2^124 (S = the largest exponent)
bool poly_block_ok(const PolyCoef& pc) {
  if (pc.E >> 24) return false;
  int32_t sj[3], S = 0;
  for (int j = 0; j < 3; j++) {
    sj[j] = (int32_t)((pc.E >> (8 * j)) & 0xFF);
    if (sj[j] > 62) return false;
    S = sj[j] > S ? sj[j] : S;
  }
  const int32_t room[3] = {49, 34, 20};
  for (int j = 0; j < 3; j++) {
    const int64_t k = pc.K[j];
    if (k > (1ll << 61) || k < -(1ll << 61)) return false;
    if (k && S - sj[j] > room[j]) return false;
  }
  return true;
}

// host-side consistency of records/starts/words (everything a kernel indexes with)
bool validate_host(const BlobHeader& h, const Record* rec, const uint64_t* starts,
                   const uint64_t* words) {
  uint64_t off = 0;
  for (uint64_t p = 0; p < h.m; p++) {
    const Record& r = rec[p];
    const bool pl = w3_poly(r.word3) != 0;
    uint64_t t0 = 0, t1 = 0;
    memcpy(&t0, &r.theta0, 8);
    memcpy(&t1, &r.theta1, 8);
    if (pl && (h.model != LECO_MODEL_POLY || w3_exact(r.word3) || w3_s(r.word3) != 0 || t0 || t1)) return false;
    const uint32_t b = w3_b(r.word3);
    if (b > 64) return false;
    const uint64_t a = r.start;
    uint64_t e;
    if (h.kind == LECO_PART_FIXED) {
      if (a != p * (uint64_t)h.L) return false;
      e = a + h.L < h.n ? a + h.L : h.n;
    } else {
      if (starts[p] != a || starts[p + 1] <= a) return false;
      e = starts[p + 1];
    }
    if (e <= a || e - a > kMaxPartLen) return false;
    if (w3_off(r.word3) != off) return false;
    if (pl) {
      if (e - a < kPolyMinLen || e - a > kPolyMaxLen) return false;
      if (off + kPolyBlockBits > 64 * (h.nwords - 1)) return false;
      if (!poly_block_ok(host_poly_block(words, off))) return false;
      off += kPolyBlockBits;
    }
    off += (e - a) * b;
    if (off >= (1ull << 48)) return false;
  }
  if (h.kind == LECO_PART_VAR && (starts[0] != 0 || starts[h.m] != h.n)) return false;
  if (h.kind == LECO_PART_FIXED && h.m != (h.n + h.L - 1) / h.L) return false;
  if (off != h.total_bits || h.nwords != stream_words(off)) return false;
  for (uint64_t w = (off + 63) / 64; w < h.nwords; w++)
    if (words[w]) return false;  // padding must be zero
  if (off % 64 && (words[off / 64] >> (off % 64))) return false;
  return true;
}

}  // namespace

namespace leco {

cudaError_t dev_alloc(void** p, uint64_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = pool_for_current_device();
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

}  // namespace leco

extern "C" {

leco_status leco_search_partition_size(const void* d_values, uint64_t n, leco_dtype dtype, leco_model model,
                                       uint32_t max_len, double sample_frac, uint64_t seed, leco_stream_t stream,
                                       uint32_t* best_L, uint64_t* best_bits, uint64_t* evals) {
  NvtxRange nvtx_range("leco_search_partition_size");
  if (!best_L || (n && !d_values) || !valid_dtype(dtype) || !valid_model(model)) return LECO_ERR_INVALID_ARG;
  if (max_len == 0) max_len = 10000;
  if (sample_frac == 0.0) sample_frac = 0.01;
  if (max_len > 16384 || !(sample_frac > 0.0 && sample_frac <= 1.0)) return LECO_ERR_INVALID_ARG;
  uint64_t bits = 0, ne = 0;
  const cudaError_t e = search_partition_size(d_values, dtype, n, sizing_model(model), max_len, sample_frac, seed,
                                              best_L, &bits, &ne, (cudaStream_t)stream);
  if (e != cudaSuccess) return from_cuda(e);
  if (best_bits) *best_bits = bits;
  if (evals) *evals = ne;
  return LECO_OK;
}

leco_status leco_selftest_wait_timeout(uint32_t limit_us, leco_stream_t stream) {
  if (limit_us < 1 || limit_us > 1000000) return LECO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* d = nullptr;
  cudaError_t e = dev_alloc((void**)&d, 4, st);
  if (e != cudaSuccess) return from_cuda(e);
  uint32_t flags = 0;
  e = cudaMemsetAsync(d, 0, 4, st);
  if (e == cudaSuccess) e = launch_wait_selftest((uint64_t)limit_us * 1000ull, d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, d, 4, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  return (flags & kStatTimeout) ? LECO_ERR_TIMEOUT : LECO_OK;
}

leco_status leco_trim_memory(void) {
  cudaMemPool_t pool = pool_for_current_device();
  if (!pool) return LECO_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return LECO_ERR_CUDA;
  return from_cuda(cudaMemPoolTrimTo(pool, 0));
}


const char* leco_status_string(leco_status s) {
  switch (s) {
    case LECO_OK: return "LECO_OK";
    case LECO_ERR_INVALID_ARG: return "LECO_ERR_INVALID_ARG";
    case LECO_ERR_OOM: return "LECO_ERR_OOM";
    case LECO_ERR_INDEX_RANGE: return "LECO_ERR_INDEX_RANGE";
    case LECO_ERR_CUDA: return "LECO_ERR_CUDA";
    case LECO_ERR_CORRUPT: return "LECO_ERR_CORRUPT";
    case LECO_ERR_TIMEOUT: return "LECO_ERR_TIMEOUT";
    case LECO_ERR_BUDGET: return "LECO_ERR_BUDGET";
  }
  return "LECO_ERR_UNKNOWN";
}

uint32_t leco_version(void) { return 10000u; }

leco_status leco_var_partition(const void* d_values, uint64_t n, leco_dtype dtype,
                               leco_partition_policy policy, leco_model model,
                               uint64_t* d_starts_out, uint64_t* m_out, leco_stream_t stream) {
  NvtxRange nvtx_range("leco_var_partition");
  if (!d_starts_out || !m_out || (n && !d_values) || !valid_dtype(dtype) || !valid_model(model))
    return LECO_ERR_INVALID_ARG;
  if ((policy.kind != LECO_PART_VAR && policy.kind != LECO_PART_VAR_SEEDED) || !(policy.tau >= 0.0 && policy.tau <= 1.0) ||
      policy.part_size > kMaxPartLen)
    return LECO_ERR_INVALID_ARG;
  const uint32_t cap = policy.part_size ? policy.part_size : kMaxPartLen;
  return from_cuda(var_partition(d_values, dtype, n, policy.tau, cap, sizing_model(model),
                                 policy.kind == LECO_PART_VAR_SEEDED, d_starts_out, m_out, (cudaStream_t)stream));
}

leco_status leco_encode(const void* d_values, uint64_t n, leco_dtype dtype,
                        leco_partition_policy policy, leco_model model, leco_stream_t stream,
                        leco_column** out) {
  NvtxRange nvtx_range("leco_encode");
  if (!out) return LECO_ERR_INVALID_ARG;
  *out = nullptr;
  if ((n && !d_values) || !valid_dtype(dtype) || !valid_model(model)) return LECO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  leco_column* c = new (std::nothrow) leco_column();
  if (!c) return LECO_ERR_OOM;
  c->n = n;
  c->dtype = dtype;
  c->model = model;
  c->kind = policy.kind;
  c->home = st;
  cudaGetDevice(&c->device);
  leco_status s = LECO_OK;
  bool encode_prefit = false;
  if (policy.kind == LECO_PART_AUTO) {  // fixed partitions of the searched size (§3.2.1)
    uint32_t L = 1;
    s = leco_search_partition_size(d_values, n, dtype, model, policy.part_size, 0.01, 0, stream, &L, nullptr,
                                   nullptr);
    if (s != LECO_OK) {
      delete c;
      return s;
    }
    policy.kind = LECO_PART_FIXED;
    policy.part_size = L;
    c->kind = LECO_PART_FIXED;
  }
  if (policy.kind == LECO_PART_FIXED) {
    if (policy.part_size < 1 || policy.part_size > kMaxPartLen) {
      delete c;
      return LECO_ERR_INVALID_ARG;
    }
    c->L = policy.part_size;
    c->m = (n + c->L - 1) / c->L;
    s = alloc_meta(c, st);
  } else if (policy.kind == LECO_PART_VAR || policy.kind == LECO_PART_VAR_SEEDED) {
    if (!(policy.tau >= 0.0 && policy.tau <= 1.0) || policy.part_size > kMaxPartLen) {
      delete c;
      return LECO_ERR_INVALID_ARG;
    }
    c->tau = policy.tau;
    c->L = 0;
    c->kind = LECO_PART_VAR;  // the seeded split gives an ordinary variable partition column
    uint64_t* tmp = nullptr;
    cudaError_t e = dev_alloc((void**)&tmp, 8 * (n + 1), st);
    if (e != cudaSuccess) {
      delete c;
      return from_cuda(e);
    }
    uint64_t m = 0;
    // the partitioner's fits are the records of a constant or linear column
    Record* prefit = nullptr;
    const uint32_t cap = policy.part_size ? policy.part_size : kMaxPartLen;
    s = from_cuda(var_partition_fit(d_values, dtype, n, policy.tau, cap, sizing_model(model),
                                    policy.kind == LECO_PART_VAR_SEEDED, tmp, &m,
                                    model == LECO_MODEL_POLY ? nullptr : &prefit, st));
    if (s == LECO_OK) {
      c->m = m;
      s = alloc_meta(c, st);
    }
    if (s == LECO_OK)
      s = from_cuda(cudaMemcpyAsync(c->starts, tmp, 8 * (m + 1), cudaMemcpyDeviceToDevice, st));
    if (s == LECO_OK && prefit && m)
      s = from_cuda(cudaMemcpyAsync(c->rec, prefit, sizeof(Record) * m, cudaMemcpyDeviceToDevice, st));
    if (s == LECO_OK) encode_prefit = prefit != nullptr;
    if (prefit) cudaFreeAsync(prefit, st);
    cudaFreeAsync(tmp, st);
  } else {
    delete c;
    return LECO_ERR_INVALID_ARG;
  }
  if (s == LECO_OK) s = encode_partitions(c, d_values, st, encode_prefit);
  if (s != LECO_OK) {
    release(c, st);
    return s;
  }
  *out = c;
  return LECO_OK;
}

leco_status leco_encode_with_starts(const void* d_values, uint64_t n, leco_dtype dtype,
                                    const uint64_t* d_starts, uint64_t m, leco_model model,
                                    leco_stream_t stream, leco_column** out) {
  NvtxRange nvtx_range("leco_encode_with_starts");
  if (!out) return LECO_ERR_INVALID_ARG;
  *out = nullptr;
  if ((n && !d_values) || !d_starts || !valid_dtype(dtype) || !valid_model(model))
    return LECO_ERR_INVALID_ARG;
  if ((n == 0) != (m == 0) || m > n) return LECO_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<uint64_t> h(m + 1);
  cudaError_t e = cudaMemcpyAsync(h.data(), d_starts, 8 * (m + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return from_cuda(e);
  if (h[0] != 0 || h[m] != n) return LECO_ERR_INVALID_ARG;
  for (uint64_t p = 0; p < m; p++)
    if (h[p + 1] <= h[p] || h[p + 1] - h[p] > kMaxPartLen) return LECO_ERR_INVALID_ARG;
  leco_column* c = new (std::nothrow) leco_column();
  if (!c) return LECO_ERR_OOM;
  c->n = n;
  c->m = m;
  c->dtype = dtype;
  c->model = model;
  c->kind = LECO_PART_VAR;
  c->home = st;
  cudaGetDevice(&c->device);
  leco_status s = alloc_meta(c, st);
  if (s == LECO_OK)
    s = from_cuda(cudaMemcpyAsync(c->starts, d_starts, 8 * (m + 1), cudaMemcpyDeviceToDevice, st));
  if (s == LECO_OK) s = encode_partitions(c, d_values, st);
  if (s != LECO_OK) {
    release(c, st);
    return s;
  }
  *out = c;
  return LECO_OK;
}

leco_status leco_decode_all(const leco_column* col, void* d_out, leco_stream_t stream) {
  NvtxRange nvtx_range("leco_decode_all");
  if (!col || (col->n && !d_out)) return LECO_ERR_INVALID_ARG;
  return from_cuda(launch_decode(view_of(col), 0, col->n, d_out, (cudaStream_t)stream));
}

leco_status leco_decode_range(const leco_column* col, uint64_t begin, uint64_t count, void* d_out,
                              leco_stream_t stream) {
  NvtxRange nvtx_range("leco_decode_range");
  if (!col || (count && !d_out) || begin > col->n || count > col->n - begin)
    return LECO_ERR_INVALID_ARG;
  return from_cuda(launch_decode(view_of(col), begin, count, d_out, (cudaStream_t)stream));
}

leco_status leco_random_access(const leco_column* col, const uint64_t* d_idx, uint64_t k,
                               void* d_out, leco_stream_t stream) {
  NvtxRange nvtx_range("leco_random_access");
  if (!col || (k && (!d_idx || !d_out))) return LECO_ERR_INVALID_ARG;
  return from_cuda(launch_random_access(view_of(col), d_idx, k, d_out, (cudaStream_t)stream));
}

leco_status leco_filter_sum(const leco_column* col, uint64_t lo, uint64_t hi, uint32_t flags,
                            leco_sum_result* d_out, leco_stream_t stream) {
  NvtxRange nvtx_range("leco_filter_sum");
  if (!col || !d_out || (flags & ~(LECO_FILTER_PRUNE | LECO_FILTER_DECODE_ALL))) return LECO_ERR_INVALID_ARG;
  return from_cuda(launch_filter_sum(view_of(col), lo, hi, flags, d_out, (cudaStream_t)stream));
}

leco_status leco_sync(const leco_column* col, leco_stream_t stream) {
  if (!col) return LECO_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  uint32_t flags = 0;
  e = cudaMemcpy(&flags, col->status, 4, cudaMemcpyDeviceToHost);
  // cleared in stream order and waited for, so a later call on any stream cannot have its flag erased
  if (e == cudaSuccess && flags) e = cudaMemsetAsync(col->status, 0, 4, (cudaStream_t)stream);
  if (e == cudaSuccess && flags) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  if (flags & kStatIndexRange) return LECO_ERR_INDEX_RANGE;
  if (flags & kStatCorrupt) return LECO_ERR_CORRUPT;
  if (flags & kStatTimeout) return LECO_ERR_TIMEOUT;
  return LECO_OK;
}

leco_status leco_stats_get(const leco_column* col, leco_stats* out) {
  if (!col || !out) return LECO_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->n = col->n;
  out->partitions = col->m;
  out->record_bytes = 32 * col->m;
  out->residual_bytes = 8 * col->nwords;
  out->total_bytes = out->record_bytes + out->residual_bytes +
                     (col->kind == LECO_PART_VAR ? 8 * (col->m + 1) : 0);
  out->ratio = col->n ? (double)out->total_bytes / (double)(col->n * value_bytes(col->dtype)) : 0.0;
  out->dtype = col->dtype;
  out->kind = col->kind;
  out->model = col->model;
  out->part_size = col->kind == LECO_PART_FIXED ? col->L : 0;
  out->residual_bits = col->total_bits;
  out->device_bytes = col->meta_bytes + col->words_bytes;
  return LECO_OK;
}

leco_status leco_column_export(const leco_column* col, void* host_records, void* host_words,
                               void* host_starts) {
  if (!col) return LECO_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(col->home);
  if (e == cudaSuccess && host_records && col->m)
    e = cudaMemcpy(host_records, col->rec, 32 * col->m, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && host_words && col->nwords)
    e = cudaMemcpy(host_words, col->words, 8 * col->nwords, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && host_starts && col->kind == LECO_PART_VAR)
    e = cudaMemcpy(host_starts, col->starts, 8 * (col->m + 1), cudaMemcpyDeviceToHost);
  return from_cuda(e);
}

leco_status leco_serialize(const leco_column* col, void* host_buf, uint64_t cap, uint64_t* bytes) {
  if (!col || !bytes) return LECO_ERR_INVALID_ARG;
  const uint64_t need = blob_bytes(col);
  *bytes = need;
  if (!host_buf) return LECO_OK;
  if (cap < need) return LECO_ERR_INVALID_ARG;
  char* b = (char*)host_buf;
  char* body = b + kHeaderBytes;
  char* p = body;
  leco_status s = leco_column_export(col, p, nullptr, nullptr);
  if (s != LECO_OK) return s;
  p += 32 * col->m;
  if (col->kind == LECO_PART_VAR) {
    s = from_cuda(cudaMemcpy(p, col->starts, 8 * (col->m + 1), cudaMemcpyDeviceToHost));
    if (s != LECO_OK) return s;
    p += 8 * (col->m + 1);
  }
  s = leco_column_export(col, nullptr, p, nullptr);
  if (s != LECO_OK) return s;
  BlobHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kMagic;
  h.version = kVersion;
  h.n = col->n;
  h.m = col->m;
  h.nwords = col->nwords;
  h.dtype = (uint8_t)col->dtype;
  h.kind = (uint8_t)col->kind;
  h.model = (uint8_t)col->model;
  h.L = col->kind == LECO_PART_FIXED ? col->L : 0;
  h.tau = col->tau;
  h.total_bits = col->total_bits;
  h.crc = crc32_update(0, body, need - kHeaderBytes);
  memcpy(b, &h, sizeof(h));
  return LECO_OK;
}

leco_status leco_deserialize(const void* host_buf, uint64_t bytes, leco_stream_t stream,
                             leco_column** out) {
  NvtxRange nvtx_range("leco_deserialize");
  if (!out || !host_buf) return LECO_ERR_INVALID_ARG;
  *out = nullptr;
  if (bytes < kHeaderBytes) return LECO_ERR_CORRUPT;
  BlobHeader h;
  memcpy(&h, host_buf, sizeof(h));
  if (h.magic != kMagic || h.version != kVersion) return LECO_ERR_CORRUPT;
  if (!valid_dtype(h.dtype) || !valid_model(h.model) ||
      (h.kind != LECO_PART_FIXED && h.kind != LECO_PART_VAR))
    return LECO_ERR_CORRUPT;
  if (h.kind == LECO_PART_FIXED && (h.L < 1 || h.L > kMaxPartLen)) return LECO_ERR_CORRUPT;
  if (h.m > h.n || (h.n > 0) != (h.m > 0) || h.nwords < 2 || h.nwords > (1ull << 42))
    return LECO_ERR_CORRUPT;
  const uint64_t need = kHeaderBytes + 32 * h.m + (h.kind == LECO_PART_VAR ? 8 * (h.m + 1) : 0) +
                        8 * h.nwords;
  if (bytes != need) return LECO_ERR_CORRUPT;
  const char* body = (const char*)host_buf + kHeaderBytes;
  if (crc32_update(0, body, need - kHeaderBytes) != h.crc) return LECO_ERR_CORRUPT;
  // records/starts/words may be unaligned inside the caller's buffer: validate on copies
  std::vector<Record> rec(h.m);
  std::vector<uint64_t> starts(h.kind == LECO_PART_VAR ? h.m + 1 : 0);
  std::vector<uint64_t> words(h.nwords);
  const char* p = body;
  if (h.m) memcpy(rec.data(), p, 32 * h.m);
  p += 32 * h.m;
  if (h.kind == LECO_PART_VAR) {
    memcpy(starts.data(), p, 8 * (h.m + 1));
    p += 8 * (h.m + 1);
  }
  memcpy(words.data(), p, 8 * h.nwords);
  if (!validate_host(h, rec.data(), starts.data(), words.data())) return LECO_ERR_CORRUPT;

  cudaStream_t st = (cudaStream_t)stream;
  leco_column* c = new (std::nothrow) leco_column();
  if (!c) return LECO_ERR_OOM;
  c->n = h.n;
  c->m = h.m;
  c->nwords = h.nwords;
  c->total_bits = h.total_bits;
  c->dtype = h.dtype;
  c->kind = h.kind;
  c->model = h.model;
  c->L = h.kind == LECO_PART_FIXED ? h.L : 0;
  c->tau = h.tau;
  c->home = st;
  for (uint64_t p = 0; p < h.m; p++) c->max_b = c->max_b > w3_b(rec[p].word3) ? c->max_b : w3_b(rec[p].word3);
  c->stage_bytes = stage_word_bytes(c->max_b) + (h.model == LECO_MODEL_POLY ? kPolyStageExtra : 0);
  // polynomial blocks, taken from the validated stream for the decode-table build
  std::vector<PolyCoef> pcoef(h.model == LECO_MODEL_POLY ? h.m : 0);
  for (uint64_t p = 0; p < pcoef.size(); p++)
    if (w3_poly(rec[p].word3)) pcoef[p] = host_poly_block(words.data(), w3_off(rec[p].word3));
  cudaGetDevice(&c->device);
  leco_status s = alloc_meta(c, st);
  if (s == LECO_OK) {
    c->words_bytes = 8 * c->nwords;
    s = from_cuda(dev_alloc((void**)&c->words, c->words_bytes, st));
  }
  if (s == LECO_OK && h.m)
    s = from_cuda(cudaMemcpyAsync(c->rec, rec.data(), 32 * h.m, cudaMemcpyHostToDevice, st));
  if (s == LECO_OK && h.kind == LECO_PART_VAR)
    s = from_cuda(cudaMemcpyAsync(c->starts, starts.data(), 8 * (h.m + 1), cudaMemcpyHostToDevice, st));
  if (s == LECO_OK)
    s = from_cuda(cudaMemcpyAsync(c->words, words.data(), 8 * h.nwords, cudaMemcpyHostToDevice, st));
  PolyCoef* d_pcoef = nullptr;
  if (s == LECO_OK && !pcoef.empty()) {
    s = from_cuda(dev_alloc((void**)&d_pcoef, sizeof(PolyCoef) * pcoef.size(), st));
    if (s == LECO_OK)
      s = from_cuda(cudaMemcpyAsync(d_pcoef, pcoef.data(), sizeof(PolyCoef) * pcoef.size(), cudaMemcpyHostToDevice, st));
  }
  if (s == LECO_OK) s = from_cuda(launch_build_aux(c->rec, d_pcoef, c->m, c->n, c->aux, c->poly, c->status, st));
  if (s == LECO_OK) s = from_cuda(launch_tile_desc(view_of(c), c->tiles, st));
  if (d_pcoef) cudaFreeAsync(d_pcoef, st);
  // the host vectors die at return: finish the copies first
  if (s == LECO_OK) s = from_cuda(cudaStreamSynchronize(st));
  if (s != LECO_OK) {
    release(c, st);
    return s;
  }
  *out = c;
  return LECO_OK;
}

void leco_column_free(leco_column* col) {
  if (!col) return;
  int prev = 0;
  const int dev = col->device;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  release(col, nullptr);
  cudaStreamSynchronize(nullptr);
  if (prev != dev) cudaSetDevice(prev);
}

void leco_column_free_async(leco_column* col, leco_stream_t stream) {
  if (!col) return;
  release(col, (cudaStream_t)stream);
}

}  // extern "C"
