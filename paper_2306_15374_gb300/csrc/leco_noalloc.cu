// Fixed-partition encode into caller-provided buffers that allocates nothing on the device.
//
// Some callers cannot call cudaMalloc: a host engine whose device memory is entirely reserved by
// its own pool (a driver allocation would fail against its cap or escape its accounting), or a
// latency-critical path where an allocation's implicit device synchronization is unacceptable.
// This entry point runs the same kernels as leco_encode's fixed-partition path, but its scratch
// (per-partition bit lengths, the offset scan, the decode table) lives in one file-scope
// __device__ array of fixed size, and the records and residual words go to the caller's buffers.
#include <mutex>

#include "leco_internal.cuh"

using namespace leco;

namespace {

// Largest partition count one call accepts (n <= 2^18 * L values).
constexpr uint64_t kNoAllocMaxParts = 1ull << 18;

// Scratch layout in 64-bit words: decode table (4 per partition, first so it is 32-byte aligned),
// bit lengths (1 per partition), offset scan (1 per partition + scan tiles + total), [total, max b].
constexpr uint64_t kScratchWords =
    4 * kNoAllocMaxParts + kNoAllocMaxParts + (kNoAllocMaxParts + kNoAllocMaxParts / 2048 + 2) + 2;

// One array per device that loads the library, held until the process exits (about 12.6 MB).
static __device__ __align__(256) uint64_t g_noalloc_scratch[kScratchWords];

std::mutex g_scratch_mu;
uint64_t* g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on the current device. In host code the array's name is only
// a host-side stand-in, so the address is looked up once per device with that device current.
leco_status scratch_for_current_device(uint64_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LECO_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LECO_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<uint64_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return LECO_OK;
}

}  // namespace

extern "C" leco_status leco_encode_fixed_noalloc(const void* d_values, uint64_t n, leco_dtype dtype,
                                                 uint32_t L, leco_model model, void* d_records,
                                                 void* d_words, uint64_t words_cap,
                                                 uint64_t* nwords_out, leco_stream_t stream) {
  if (!nwords_out) return LECO_ERR_INVALID_ARG;
  *nwords_out = 0;
  if ((dtype != LECO_U32 && dtype != LECO_U64) ||
      (model != LECO_MODEL_CONSTANT && model != LECO_MODEL_LINEAR) || L < 1 || L > kMaxPartLen)
    return LECO_ERR_INVALID_ARG;
  if ((n && (!d_values || !d_records)) || !d_words) return LECO_ERR_INVALID_ARG;
  const uint64_t m = (n + L - 1) / L;
  if (m > kNoAllocMaxParts) return LECO_ERR_INVALID_ARG;  // beyond the fixed scratch
  uint64_t* scratch = nullptr;
  leco_status s = scratch_for_current_device(&scratch);
  if (s != LECO_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  Aux* aux = reinterpret_cast<Aux*>(scratch);
  uint64_t* lenbits = scratch + 4 * kNoAllocMaxParts;
  uint64_t* off_scr = lenbits + kNoAllocMaxParts;
  uint64_t* res = off_scr + (kNoAllocMaxParts + kNoAllocMaxParts / 2048 + 2);  // [total, max b]
  Record* rec = static_cast<Record*>(d_records);
  // every scratch word this call reads is written first by this call (launch_fit zeroes max b; the
  // word after it records a staging copy that timed out)
  uint32_t* err = reinterpret_cast<uint32_t*>(res + 1) + 1;
  cudaError_t e = cudaMemsetAsync(err, 0, 4, st);
  if (e == cudaSuccess)
    e = launch_fit(d_values, dtype, n, nullptr, L, m, model, rec, lenbits, nullptr,
                   reinterpret_cast<uint32_t*>(res + 1), err, st);
  if (e == cudaSuccess) e = launch_offsets(rec, lenbits, m, off_scr, offsets_scratch_elems(m), res, st);
  uint64_t total = 0;
  uint32_t flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, res, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LECO_ERR_OOM : LECO_ERR_CUDA;
  if (flags & kStatTimeout) return LECO_ERR_TIMEOUT;
  if (total >= (1ull << 48)) return LECO_ERR_INVALID_ARG;
  const uint64_t nwords = stream_words(total);
  *nwords_out = nwords;
  if (nwords > words_cap) return LECO_ERR_INVALID_ARG;  // *nwords_out tells the size needed
  e = launch_build_aux(rec, nullptr, m, n, aux, nullptr, nullptr, st);
  if (e == cudaSuccess)
    e = launch_pack(d_values, dtype, rec, aux, nullptr, nullptr, m, n, total, static_cast<uint64_t*>(d_words), nwords,
                    err, st);
  // A staging copy that gave up leaves part of the stream unwritten, and this call has no column
  // whose status word could carry the flag to a later leco_sync: read it back here, before the
  // next call's clear can erase it.
  flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  return (flags & kStatTimeout) ? LECO_ERR_TIMEOUT : LECO_OK;
}
