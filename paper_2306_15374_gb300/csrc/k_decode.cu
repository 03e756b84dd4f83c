// Decoder kernels (§3.3 Decoder): range/full decompression, the fused filter + sum scan (§5.1's
// filter without materialising values) and batched point lookups.
//
// Value at position i of partition p: pred_p(i - start_p) + unzigzag(bits [off_p + b_p (i -
// start_p), +b_p)) mod 2^64. The prediction comes from the decode table (integer grid) and falls
// back to binary64 for records whose exact flag did not verify.
#include "leco_internal.cuh"

namespace leco {

namespace {

constexpr int kBlock = 256;
constexpr int kGroups = 8;  // 32-value groups per warp chunk

__device__ __forceinline__ uint64_t part_start(const ColumnView& c, uint64_t p) {
  if (c.starts) return __ldg(c.starts + p);
  const uint64_t s = p * (uint64_t)c.L;
  return s < c.n ? s : c.n;
}

// partition holding position i (< n): fixed i / L, variable largest p with starts[p] <= i
__device__ __forceinline__ uint64_t find_part(const ColumnView& c, uint64_t i) {
  if (!c.starts) {
    if (c.n <= 0xFFFFFFFFull) return (uint32_t)i / c.L;
    return i / c.L;
  }
  uint64_t lo = 0, hi = c.m;
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

// Walk one warp chunk of 32*kGroups consecutive positions starting at `first`; calls f(i, value)
// for every position i < end handled by this lane.
template <typename F>
__device__ __forceinline__ void walk_chunk(const ColumnView& c, uint64_t first, uint64_t end, F&& f) {
  const uint32_t lane = threadIdx.x & 31u;
  uint64_t p = find_part(c, first);
  uint64_t pend = part_start(c, p + 1);
  Aux a = load_aux(c.aux, p);
#pragma unroll
  for (int g = 0; g < kGroups; g++) {
    const uint64_t i = first + (uint64_t)g * 32 + lane;
    if (i >= end) break;
    while (i >= pend) {
      p++;
      pend = part_start(c, p + 1);
      a = load_aux(c.aux, p);
    }
    const uint64_t x = i - a.start;
    const uint32_t b = w3_b(a.word3);
    const uint64_t z = read_field(c.words, w3_off(a.word3) + x * b, b);
    const int64_t pred = predict_aux(a, c.rec, p, x);
    f(i, (uint64_t)pred + (uint64_t)zz_decode(z));
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
    k_decode(const ColumnView c, uint64_t begin, uint64_t count, T* __restrict__ out) {
  const uint64_t warp = ((uint64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kBlock) >> 5;
  const uint64_t chunk = 32ull * kGroups;
  const uint64_t end = begin + count;
  const uint64_t nchunks = (count + chunk - 1) / chunk;
  for (uint64_t ch = warp; ch < nchunks; ch += nwarps) {
    walk_chunk(c, begin + ch * chunk, end, [&](uint64_t i, uint64_t v) { out[i - begin] = (T)v; });
  }
}

// 128-bit unsigned accumulate
struct Sum128 {
  uint64_t lo, hi;
  __device__ __forceinline__ void add(uint64_t v) {
    const uint64_t t = lo + v;
    hi += (t < lo) ? 1ull : 0ull;
    lo = t;
  }
};

__device__ __forceinline__ Sum128 warp_sum128(Sum128 s) {
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t l2 = __shfl_down_sync(0xffffffffu, s.lo, o);
    const uint64_t h2 = __shfl_down_sync(0xffffffffu, s.hi, o);
    const uint64_t nl = s.lo + l2;
    s.hi = s.hi + h2 + (nl < s.lo ? 1ull : 0ull);
    s.lo = nl;
  }
  return s;
}

__global__ void __launch_bounds__(kBlock)
    k_filter_sum(const ColumnView c, uint64_t lo, uint64_t hi, leco_sum_result* __restrict__ out) {
  const uint64_t warp = ((uint64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * kBlock) >> 5;
  const uint64_t chunk = 32ull * kGroups;
  const uint64_t nchunks = (c.n + chunk - 1) / chunk;
  const uint64_t vmask = c.dtype == LECO_U32 ? 0xFFFFFFFFull : ~0ull;
  uint64_t cnt = 0;
  Sum128 sum{0, 0};
  for (uint64_t ch = warp; ch < nchunks; ch += nwarps) {
    walk_chunk(c, ch * chunk, c.n, [&](uint64_t, uint64_t v) {
      v &= vmask;
      if (v >= lo && v <= hi) {
        cnt++;
        sum.add(v);
      }
    });
  }
  cnt = warp_sum_u64(cnt);
  sum = warp_sum128(sum);
  __shared__ uint64_t s_cnt[kBlock / 32], s_lo[kBlock / 32], s_hi[kBlock / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_cnt[wid] = cnt;
    s_lo[wid] = sum.lo;
    s_hi[wid] = sum.hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Sum128 t{0, 0};
    uint64_t tc = 0;
    for (int k = 0; k < kBlock / 32; k++) {
      tc += s_cnt[k];
      const uint64_t nl = t.lo + s_lo[k];
      t.hi += s_hi[k] + (nl < t.lo ? 1ull : 0ull);
      t.lo = nl;
    }
    if (tc) {
      atomicAdd((unsigned long long*)&out->count, (unsigned long long)tc);
      const unsigned long long old = atomicAdd((unsigned long long*)&out->sum_lo, (unsigned long long)t.lo);
      const uint64_t carry = (old + t.lo < old) ? 1ull : 0ull;
      if (t.hi + carry) atomicAdd((unsigned long long*)&out->sum_hi, (unsigned long long)(t.hi + carry));
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
    k_random_access(const ColumnView c, const uint64_t* __restrict__ idx, uint64_t k,
                    T* __restrict__ out) {
  for (uint64_t q = (uint64_t)blockIdx.x * kBlock + threadIdx.x; q < k;
       q += (uint64_t)gridDim.x * kBlock) {
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
    const int64_t pred = predict_aux(a, c.rec, p, x);
    out[q] = (T)((uint64_t)pred + (uint64_t)zz_decode(z));
  }
}

int grid_for(uint64_t items, int per_block, int max_blocks_per_sm) {
  const uint64_t need = (items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)sm_count() * max_blocks_per_sm;
  return (int)(need < cap ? (need ? need : 1) : cap);
}

}  // namespace

cudaError_t launch_decode(const ColumnView& c, uint64_t begin, uint64_t count, void* out,
                          cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const int grid = grid_for((count + 32ull * kGroups - 1) / (32ull * kGroups) * 32, kBlock, 8);
  if (c.dtype == LECO_U32)
    k_decode<uint32_t><<<grid, kBlock, 0, st>>>(c, begin, count, (uint32_t*)out);
  else
    k_decode<uint64_t><<<grid, kBlock, 0, st>>>(c, begin, count, (uint64_t*)out);
  return cudaGetLastError();
}

cudaError_t launch_filter_sum(const ColumnView& c, uint64_t lo, uint64_t hi, uint32_t flags,
                              leco_sum_result* out, cudaStream_t st) {
  (void)flags;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(leco_sum_result), st);
  if (e != cudaSuccess || c.n == 0 || lo > hi) return e;
  const int grid = grid_for((c.n + 32ull * kGroups - 1) / (32ull * kGroups) * 32, kBlock, 8);
  k_filter_sum<<<grid, kBlock, 0, st>>>(c, lo, hi, out);
  return cudaGetLastError();
}

cudaError_t launch_random_access(const ColumnView& c, const uint64_t* idx, uint64_t k, void* out,
                                 cudaStream_t st) {
  if (k == 0) return cudaSuccess;
  const int grid = grid_for(k, kBlock, 8);
  if (c.dtype == LECO_U32)
    k_random_access<uint32_t><<<grid, kBlock, 0, st>>>(c, idx, k, (uint32_t*)out);
  else
    k_random_access<uint64_t><<<grid, kBlock, 0, st>>>(c, idx, k, (uint64_t*)out);
  return cudaGetLastError();
}

}  // namespace leco
