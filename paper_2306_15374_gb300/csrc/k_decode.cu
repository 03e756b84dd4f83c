// Batched point lookups (§3.3 Decoder): one thread per requested position.
//
// Value at position i of partition p: pred_p(i - start_p) + unzigzag(bits [off_p + b_p (i -
// start_p), +b_p)) mod 2^64. The prediction comes from the decode table (integer grid) and falls
// back to binary64 for records whose exact flag did not verify.
#include "leco_internal.cuh"

namespace leco {

namespace {

constexpr int kBlock = 256;

// partition holding position i (< n): fixed i / L; variable: largest p with starts[p] <= i, searched
// among the partitions touching i's scan tile (its descriptor names the first and how many), so a
// lookup costs one descriptor load and a search over a few starts instead of over all of them
__device__ __forceinline__ uint64_t find_part(const ColumnView& c, uint64_t i) {
  if (!c.starts) {
    if (c.n <= 0xFFFFFFFFull) return (uint32_t)i / c.L;
    return i / c.L;
  }
  const TileDesc* d = c.tiles + i / kScanTile;
  uint64_t lo = __ldg(&d->p0), hi = lo + __ldg(&d->np);
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(c.starts + mid) <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ Aux load_aux(const Aux* __restrict__ aux, uint64_t p) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(aux + p);
  const ulonglong2 v0 = __ldg(q), v1 = __ldg(q + 1);
  Aux a;
  a.A = (int64_t)v0.x;
  a.B = (int64_t)v0.y;
  a.start = v1.x;
  a.word3 = v1.y;
  return a;
}

// kUnroll independent lookups per thread and iteration: their loads (index, decode-table entry,
// residual words) are issued together, so each thread keeps several memory round trips in flight.
constexpr int kUnroll = 4;

template <typename T>
__global__ void __launch_bounds__(kBlock)
    k_random_access(const ColumnView c, const uint64_t* __restrict__ idx, uint64_t k,
                    T* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * kBlock;
  for (uint64_t base = (uint64_t)blockIdx.x * kBlock + threadIdx.x; base < k; base += stride * kUnroll) {
    uint64_t i[kUnroll], p[kUnroll];
    bool ok[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const uint64_t q = base + (uint64_t)u * stride;
      i[u] = q < k ? __ldg(idx + q) : 0;
      ok[u] = q < k && i[u] < c.n;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) p[u] = ok[u] ? find_part(c, i[u]) : 0;
    Aux a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) a[u] = load_aux(c.aux, ok[u] ? p[u] : 0);
    uint64_t z[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const uint64_t x = i[u] - a[u].start;
      const uint32_t b = w3_b(a[u].word3);
      z[u] = ok[u] ? read_field(c.words, w3_off(a[u].word3) + x * b, b) : 0;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; u++) {
      const uint64_t q = base + (uint64_t)u * stride;
      if (q >= k) continue;
      if (!ok[u]) {
        out[q] = 0;
        atomicOr(c.status, kStatIndexRange);
        continue;
      }
      const int64_t pred = predict_aux(a[u], c.rec, c.poly, p[u], i[u] - a[u].start);
      out[q] = (T)((uint64_t)pred + (uint64_t)zz_decode(z[u]));
    }
  }
}

// Lookups of several columns in one launch (a serving batch): index q reads column col[q]; results
// are widened to 64 bits (a 32-bit column's value is zero-extended).
__global__ void __launch_bounds__(kBlock)
    k_lookup_multi(const ColumnView* __restrict__ views, const uint32_t* __restrict__ col,
                   const uint64_t* __restrict__ idx, uint64_t k, uint64_t* __restrict__ out) {
  for (uint64_t q = (uint64_t)blockIdx.x * kBlock + threadIdx.x; q < k; q += (uint64_t)gridDim.x * kBlock) {
    const ColumnView c = views[col[q]];
    const uint64_t i = __ldg(idx + q);
    if (i >= c.n) {
      out[q] = 0;
      atomicOr(c.status, kStatIndexRange);
      continue;
    }
    const uint64_t p = find_part(c, i);
    const Aux a = load_aux(c.aux, p);
    const uint64_t x = i - a.start;
    const uint32_t b = w3_b(a.word3);
    const uint64_t z = read_field(c.words, w3_off(a.word3) + x * b, b);
    const uint64_t v = (uint64_t)predict_aux(a, c.rec, c.poly, p, x) + (uint64_t)zz_decode(z);
    out[q] = c.dtype == LECO_U32 ? (v & 0xFFFFFFFFull) : v;
  }
}

int grid_for(uint64_t items, int per_block, int max_blocks_per_sm) {
  const uint64_t need = (items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)sm_count() * max_blocks_per_sm;
  return (int)(need < cap ? (need ? need : 1) : cap);
}

}  // namespace

cudaError_t launch_random_access(const ColumnView& c, const uint64_t* idx, uint64_t k, void* out,
                                 cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  const int grid = grid_for((k + kUnroll - 1) / kUnroll, kBlock, 8);
  if (c.dtype == LECO_U32)
    k_random_access<uint32_t><<<grid, kBlock, 0, st>>>(c, idx, k, (uint32_t*)out);
  else
    k_random_access<uint64_t><<<grid, kBlock, 0, st>>>(c, idx, k, (uint64_t*)out);
  return cudaGetLastError();
}

cudaError_t launch_lookup_multi(const ColumnView* views, const uint32_t* col, const uint64_t* idx, uint64_t k,
                                uint64_t* out, cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  k_lookup_multi<<<grid_for(k, kBlock, 8), kBlock, 0, st>>>(views, col, idx, k, out);
  return cudaGetLastError();
}

}  // namespace leco
