// Throughput probes of the execution units the scan, fit and partitioner kernels lean on, so that
// a kernel's "instruction-bound" can be stated against a measured number on the device at hand
// (the paper has no counterpart: it measures on CPUs). Each probe runs many independent chains of
// one kind of operation in every thread of a full grid and times them with CUDA events.
#include "leco_internal.cuh"

namespace leco {
namespace {

constexpr int kProbeChains = 8;  // independent accumulators per thread
constexpr int kProbeBlock = 256;

// KIND 0: x = (x ^ (x >> 7)) + c in 32 bits (three integer operations per step: shift, xor, add);
// 1: the same in 64 bits (three 64-bit operations); 2: x = funnel-shift-right(x, y, x & 31) with y
// the next chain (two operations: and, funnel shift); 3: binary64 multiply then add (two, no FMA).
// Every step depends on the previous value through a non-linear map, so no chain can be folded or
// shortened; the result is stored when the (run-time, always zero in practice) flag store is set,
// which the compiler cannot know.
template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) k_probe(uint64_t iters, uint32_t seed, uint32_t store, uint64_t* sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t out = 0;
  if (KIND == 0) {
    uint32_t a[kProbeChains];
    const uint32_t c = seed * 2654435761u + 1u;
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) a[u] = t * (u + 3) + seed;
    for (uint64_t i = 0; i < iters; i++) {
#pragma unroll
      for (int u = 0; u < kProbeChains; u++) a[u] = (a[u] ^ (a[u] >> 7)) + c;
    }
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) out += a[u];
  } else if (KIND == 1) {
    uint64_t a[kProbeChains];
    const uint64_t c = (uint64_t)seed * 0x9E3779B97F4A7C15ull + 1u;
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) a[u] = (uint64_t)t * (u + 3) + seed;
    for (uint64_t i = 0; i < iters; i++) {
#pragma unroll
      for (int u = 0; u < kProbeChains; u++) a[u] = (a[u] ^ (a[u] >> 13)) + c;
    }
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) out += a[u];
  } else if (KIND == 2) {
    uint32_t a[kProbeChains];
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) a[u] = t * (u + 3) + seed;
    for (uint64_t i = 0; i < iters; i++) {
#pragma unroll
      for (int u = 0; u < kProbeChains; u++) a[u] = __funnelshift_r(a[u], a[(u + 1) % kProbeChains], a[u] & 31u);
    }
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) out += a[u];
  } else {
    double a[kProbeChains];
    const double m = 1.0000001 + 1e-9 * (double)(seed & 7u), c = 1e-7 * (double)((t & 15u) + 1u);
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) a[u] = (double)(t + u);
    for (uint64_t i = 0; i < iters; i++) {
#pragma unroll
      for (int u = 0; u < kProbeChains; u++) a[u] = __dadd_rn(__dmul_rn(a[u], m), c);
    }
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) out += (uint64_t)(int64_t)a[u];
  }
  if (store) sink[t] = out;
}

// KIND 4: random 8-byte reads from a buffer far larger than L2 (nwords words): each step every
// chain reads the word at a SplitMix64-scattered index that depends on the previous word read, so
// the reads of one chain are serial and the chains of all threads are independent; the rate is one
// random DRAM sector per read.
__global__ void __launch_bounds__(kProbeBlock) k_probe_gather(const uint64_t* __restrict__ buf, uint64_t nwords,
                                                               uint64_t iters, uint32_t seed, uint32_t store,
                                                               uint64_t* sink) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t h[kProbeChains];
#pragma unroll
  for (int u = 0; u < kProbeChains; u++) h[u] = splitmix64(t * kProbeChains + u + ((uint64_t)seed << 40));
  for (uint64_t i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < kProbeChains; u++) h[u] = splitmix64(h[u] ^ __ldg(buf + (h[u] % nwords)));
  }
  uint64_t out = 0;
#pragma unroll
  for (int u = 0; u < kProbeChains; u++) out += h[u];
  if (store) sink[t] = out;
}

template <int KIND>
cudaError_t run_probe(uint64_t iters, uint32_t seed, uint64_t* sink, int blocks, cudaStream_t st) {
  k_probe<KIND><<<blocks, kProbeBlock, 0, st>>>(iters, seed, 0u, sink);
  return cudaGetLastError();
}

cudaError_t probe_launch(int kind, uint64_t iters, uint32_t seed, uint64_t* sink, int blocks, cudaStream_t st) {
  switch (kind) {
    case 0: return run_probe<0>(iters, seed, sink, blocks, st);
    case 1: return run_probe<1>(iters, seed, sink, blocks, st);
    case 2: return run_probe<2>(iters, seed, sink, blocks, st);
    default: return run_probe<3>(iters, seed, sink, blocks, st);
  }
}

}  // namespace
}  // namespace leco

using namespace leco;

namespace {

// kind 4: random gathers from a 2 GiB buffer (zeroed: the reads' values do not matter)
leco_status probe_gather(double* ops_per_s, cudaStream_t st) {
  const uint64_t nwords = (2ull << 30) / 8;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_probe_gather, kProbeBlock, 0) != cudaSuccess)
    return LECO_ERR_CUDA;
  const int blocks = sm_count() * (nb > 0 ? nb : 1);
  uint64_t* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = dev_alloc((void**)&buf, 8 * nwords, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 8 * nwords, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const uint64_t iters = 64;
  if (e == cudaSuccess) {
    k_probe_gather<<<blocks, kProbeBlock, 0, st>>>(buf, nwords, iters / 8, 1, 0u, buf);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) {
    k_probe_gather<<<blocks, kProbeBlock, 0, st>>>(buf, nwords, iters, 2, 0u, buf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (buf) cudaFreeAsync(buf, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  const double reads = (double)kProbeChains * (double)iters * (double)blocks * kProbeBlock;
  *ops_per_s = ms > 0.f ? reads / (ms * 1e-3) : 0.0;
  return LECO_OK;
}

}  // namespace

extern "C" leco_status leco_probe_throughput(int32_t kind, double* ops_per_s, leco_stream_t stream) {
  if (!ops_per_s || kind < 0 || kind > 4) return LECO_ERR_INVALID_ARG;
  *ops_per_s = 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  if (kind == 4) return probe_gather(ops_per_s, st);
  int nb = 0;
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_probe<0>, kProbeBlock, 0); break;
    case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_probe<1>, kProbeBlock, 0); break;
    case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_probe<2>, kProbeBlock, 0); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_probe<3>, kProbeBlock, 0); break;
  }
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  const int blocks = sm_count() * (nb > 0 ? nb : 1);
  uint64_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = dev_alloc((void**)&sink, 8, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // the binary64 units are far narrower than the integer ones: fewer steps keep every probe short
  const uint64_t iters = kind == 3 ? 2000 : 20000;
  if (e == cudaSuccess) e = probe_launch(kind, iters / 10, 1, sink, blocks, st);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = probe_launch(kind, iters, 2, sink, blocks, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (sink) cudaFreeAsync(sink, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return LECO_ERR_CUDA;
  const double per_step = kind <= 1 ? 3.0 : 2.0;
  const double ops = per_step * (double)kProbeChains * (double)iters * (double)blocks * kProbeBlock;
  *ops_per_s = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
  return LECO_OK;
}
