// Variable-length partitioning on the GPU (§3.2.2): split, then merge.
//
// Split: the sequence is cut into chunks of kChunk values (chunk edges always start a partition);
// inside a chunk partitions grow left to right: v_j joins the open partition [i, j) iff
// C = (j+1-i) D(v[i,j+1)) - (j-i) D(v[i,j)) <= tau * S_M and j - i < cap, where D is the linear
// regressor's fast metric bitlen(max d - min d) over the inner differences d_k = w_k - w_{k-1}. A
// warp takes a chunk and tests 32 candidates per step (prefix scans of the extremes, a ballot for
// the first refusal). Starts go to a bitmap (each warp owns its chunk's words), then a popcount
// scan compacts them.
//
// Merge, round-synchronous: each round computes for every adjacent pair the size of the merged
// partition with the full regressor (S_M + len * b) and its gain over the two apart; every pair
// with a positive gain whose priority (gain, SplitMix64 of its start) beats both neighbouring
// pairs merges, all at once. Rounds repeat until none merges. Pair sizes are cached: only pairs
// touching a partition merged in the previous round are refitted, and a refit needs one pass over
// the pair's values, because every partition carries the moments of its values and two
// partitions' moments combine exactly (see SpanStats). The fits of the final partitions are the
// column's records, so the encoder does not fit them again.
#include <math.h>

#include <map>
#include <type_traits>
#include <vector>

#include "fit.cuh"
#include "leco_internal.cuh"
#include "span_fit.cuh"
#include "var_partition.cuh"

namespace leco {

cudaError_t scan_u64(const uint64_t* in, uint64_t count, uint64_t* out, uint64_t* scratch,
                     uint64_t* total, cudaStream_t st);

namespace {

constexpr uint64_t kChunk = 1ull << 16;
constexpr uint8_t kChunkNarrow = 1, kChunkLanes = 2;  // chunk classes (k_chunk_class)
constexpr uint32_t kClassSample = 8192;               // positions per chunk that estimate its cut density,
constexpr uint32_t kClassWindows = 8;                 // in this many windows spread over the chunk
constexpr uint64_t kNone = ~0ull;  // no merged size (pair longer than the cap)

// One greedy step of the split at position j with value w (the previous value prev): returns true
// when v_j joins the open partition [i, j). NARROW: the chunk's values lie in (-2^62, 2^62) as
// int64, so differences and their running extremes fit 64 bits (their range below 2^64, taken
// unsigned); otherwise 128-bit. The threshold test C <= tau S_M is done on integers: for an integer
// C and a real t, C <= t exactly when C <= floor(t).
template <typename D>
__device__ __forceinline__ bool split_step(uint64_t j, int64_t w, int64_t prev, uint64_t& i, D& dmax, D& dmin,
                                           int& cur, uint32_t cap, int64_t tfloor) {
  bool take = (j - i) < cap;
  D nmax = dmax, nmin = dmin;
  int next = 0;
  if (take) {
    const D d = (D)w - (D)prev;
    if (j == i + 1) {
      nmax = d;
      nmin = d;
    } else {
      nmax = d > nmax ? d : nmax;
      nmin = d < nmin ? d : nmin;
    }
    if (std::is_same<D, int64_t>::value)
      next = bitlen_u64((uint64_t)nmax - (uint64_t)nmin);
    else
      next = bitlen_u128((u128)(nmax - nmin));
    const int64_t C = (int64_t)(j + 1 - i) * next - (int64_t)(j - i) * cur;
    take = C <= tfloor;
  }
  if (take) {
    cur = next;
    dmax = nmax;
    dmin = nmin;
  } else {
    i = j;
    cur = 0;
    dmax = 0;
    dmin = 0;
  }
  return take;
}

// One step of the same rule for a narrow chunk, with positions relative to the chunk (below 2^17)
// so that the cost C stays in 32 bits: a chunk's partition is at most 2^16 long and D <= 64, so
// |C| < 2^23, and tf32 = min(floor(tau S_M), 2^31 - 1) decides C <= tau S_M exactly.
__device__ __forceinline__ bool split_step_narrow(uint32_t jj, int64_t d, uint32_t& ii, int64_t& dmax, int64_t& dmin,
                                                  int& cur, uint32_t cap, int32_t tf32) {
  const uint32_t len = jj - ii;
  int64_t nmax = max(dmax, d), nmin = min(dmin, d);
  if (len == 1) nmax = nmin = d;
  const int next = bitlen_u64((uint64_t)nmax - (uint64_t)nmin);
  const int32_t C = (int32_t)(len + 1) * next - (int32_t)len * cur;
  const bool take = len < cap && C <= tf32;
  cur = take ? next : 0;
  dmax = take ? nmax : 0;
  dmin = take ? nmin : 0;
  ii = take ? ii : jj;
  return take;
}

// Left-to-right split of 32 chunks per warp (lane l sweeps chunk 32 w + l), for the chunks whose
// class has kChunkLanes (dense cuts, or values beyond the narrow range); a warp without such a
// chunk returns at once. Segment k of every chunk (positions k kSplitSeg .. + kSplitSeg) is loaded
// by the whole warp with coalesced loads one segment ahead, transposed through shared memory (row x
// holds position x of the 32 chunks, padded against bank conflicts), and then swept by each lane
// from shared memory while the next segment's loads are in flight. A segment is one bitmap word per
// chunk.
constexpr uint32_t kSplitSeg = 64;

template <typename T>
__global__ void __launch_bounds__(32) k_split_lanes(const T* __restrict__ v, uint64_t n, uint32_t cap, int64_t tfloor,
                                                    const uint8_t* __restrict__ cls, uint64_t* __restrict__ bitmap) {
  __shared__ T ring[2][kSplitSeg][33];
  const uint32_t lane = threadIdx.x;
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  const uint64_t c0 = (uint64_t)blockIdx.x * 32;
  const uint64_t c = c0 + lane;
  const bool has = c < nchunks && (cls[c] & kChunkLanes);
  if (!__any_sync(0xffffffffu, has)) return;
  const uint64_t a = c * kChunk;
  const uint32_t clen = has ? (uint32_t)(min(a + kChunk, n) - a) : 0u;  // the chunk's values
  const bool nar = has ? (cls[c] & kChunkNarrow) != 0 : true;
  const int32_t tf32 = tfloor > (int64_t)INT32_MAX ? INT32_MAX : (int32_t)tfloor;
  constexpr uint32_t nseg = (uint32_t)(kChunk / kSplitSeg);
  T r[kSplitSeg];
#pragma unroll
  for (uint32_t u = 0; u < kSplitSeg; u++) {  // segment 0 (two loads per chunk)
    const uint32_t cc = u >> 1, x = ((u & 1u) << 5) + lane;
    const uint64_t pos = (c0 + cc) * kChunk + x;
    r[u] = pos < n ? __ldg(v + pos) : (T)0;
  }
#pragma unroll
  for (uint32_t u = 0; u < kSplitSeg; u++) ring[0][((u & 1u) << 5) + lane][u >> 1] = r[u];
  __syncwarp();
  uint32_t ii = 0;  // open partition [ii, jj) relative to the chunk
  uint64_t iw = a;  // the same, absolute (wide chunks)
  int64_t prev = has ? (int64_t)ring[0][0][lane] : 0;
  int64_t dmax64 = 0, dmin64 = 0;
  i128 dmax128 = 0, dmin128 = 0;
  int cur = 0;
  for (uint32_t k = 0; k < nseg; k++) {
    const uint32_t slot = k & 1u;
    if (k + 1 < nseg) {  // issue segment k + 1
#pragma unroll
      for (uint32_t u = 0; u < kSplitSeg; u++) {
        const uint32_t cc = u >> 1, x = ((u & 1u) << 5) + lane;
        const uint64_t pos = (c0 + cc) * kChunk + (uint64_t)(k + 1) * kSplitSeg + x;
        r[u] = pos < n ? __ldg(v + pos) : (T)0;
      }
    }
    const uint32_t base = k * kSplitSeg;
    if (base < clen) {
      uint64_t word = k == 0 ? 1ull : 0ull;  // the chunk's first position opens a partition
      const uint32_t x0 = k == 0 ? 1u : 0u;
      const uint32_t xe = clen - base < kSplitSeg ? clen - base : kSplitSeg;
      bool d32 = false;  // a whole segment whose differences, and the open partition's extremes, fit int32
      if (nar && x0 == 0 && xe == kSplitSeg) {
        d32 = dmax64 >= INT32_MIN && dmax64 <= INT32_MAX && dmin64 >= INT32_MIN && dmin64 <= INT32_MAX;
        int64_t p = prev;
#pragma unroll 8
        for (uint32_t x = 0; x < kSplitSeg; x++) {
          const int64_t w = (int64_t)ring[slot][x][lane];
          const int64_t d = w - p;
          d32 = d32 && d >= INT32_MIN && d <= INT32_MAX;
          p = w;
        }
      }
      if (d32) {
        // the same steps in 32 bits: the extremes' difference stays below 2^32, so its bit length
        // (and every decision) is that of the 64-bit step
        int32_t mx = (int32_t)dmax64, mn = (int32_t)dmin64;
        uint32_t pw = (uint32_t)prev;
#pragma unroll 8
        for (uint32_t x = 0; x < kSplitSeg; x++) {
          const uint32_t w = (uint32_t)ring[slot][x][lane];
          const int32_t d = (int32_t)(w - pw);
          pw = w;
          const uint32_t len = base + x - ii;
          int32_t nmax = max(mx, d), nmin = min(mn, d);
          if (len == 1) nmax = nmin = d;
          const int next = 32 - __clz((int)((uint32_t)nmax - (uint32_t)nmin));
          const int32_t C = (int32_t)(len + 1) * next - (int32_t)len * cur;
          const bool take = len < cap && C <= tf32;
          cur = take ? next : 0;
          mx = take ? nmax : 0;
          mn = take ? nmin : 0;
          ii = take ? ii : base + x;
          if (!take) word |= 1ull << x;
        }
        dmax64 = mx;
        dmin64 = mn;
        prev = (int64_t)ring[slot][kSplitSeg - 1][lane];
      } else if (nar && x0 == 0 && xe == kSplitSeg) {
        // a whole segment: unrolled, so that the shared-memory reads run ahead of the step chain
#pragma unroll 8
        for (uint32_t x = 0; x < kSplitSeg; x++) {
          const int64_t w = (int64_t)ring[slot][x][lane];
          if (!split_step_narrow(base + x, w - prev, ii, dmax64, dmin64, cur, cap, tf32)) word |= 1ull << x;
          prev = w;
        }
      } else if (nar) {
        for (uint32_t x = x0; x < xe; x++) {
          const int64_t w = (int64_t)ring[slot][x][lane];
          if (!split_step_narrow(base + x, w - prev, ii, dmax64, dmin64, cur, cap, tf32)) word |= 1ull << x;
          prev = w;
        }
      } else {
        for (uint32_t x = x0; x < xe; x++) {
          const int64_t w = (int64_t)ring[slot][x][lane];
          if (!split_step<i128>(a + base + x, w, prev, iw, dmax128, dmin128, cur, cap, tfloor)) word |= 1ull << x;
          prev = w;
        }
      }
      bitmap[(a + base) >> 6] = word;
    }
    __syncwarp();
    if (k + 1 < nseg) {
#pragma unroll
      for (uint32_t u = 0; u < kSplitSeg; u++) ring[slot ^ 1u][((u & 1u) << 5) + lane][u >> 1] = r[u];
      __syncwarp();
    }
  }
}

// Warp-cooperative split, a warp per chunk, with the result of split_step's left-to-right sweep. From
// the open partition [i, j0) the warp tests the 32 candidates j = j0 .. j0 + 31 at once, lane l
// assuming that every candidate before it joined: the running extremes of the differences are the
// carried ones combined with an inclusive max / min scan over the lanes, the fast metric of [i, j)
// is the previous lane's metric of [i, j + 1) (the carried one for lane 0), and C follows as in
// split_step, in 32 bits: a chunk's partition is at most 2^16 long and the metric at most 64, so
// |C| < 2^23, and tf32 = min(floor(tau S_M), 2^31 - 1) decides C <= tau S_M exactly. The first
// refused candidate (a ballot) opens the next partition and the warp
// restarts after it; when none is refused the last lane's state carries over 32 positions on. A
// partition of length len costs about len / 32 + 1 steps instead of len dependent steps, which pays
// where partitions are long: the chunks whose class lacks kChunkLanes (narrow, few cuts). The warp
// stages its chunk through a two-block shared-memory ring, one block of loads ahead.
constexpr uint32_t kSplitWarps = 4;
constexpr uint32_t kSplitBlk = 256;  // values per staged block (8 per lane)

// bitmap must be zero on entry: a warp stores only its chunk's words that hold a start
template <typename T>
__global__ void __launch_bounds__(32 * kSplitWarps)
    k_split_warp(const T* __restrict__ v, uint64_t n, uint32_t cap, int64_t tfloor, const uint8_t* __restrict__ cls,
                 uint64_t* __restrict__ bitmap) {
  constexpr uint32_t kRing = 2 * kSplitBlk, kMask = kRing - 1;
  __shared__ T ring[kSplitWarps][kRing];
  const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  const uint64_t c = (uint64_t)blockIdx.x * kSplitWarps + wid;
  if (c >= nchunks || (cls[c] & kChunkLanes)) return;  // the whole warp: no block-wide barrier follows
  const uint64_t a = c * kChunk;
  const uint32_t clen = (uint32_t)(min(a + kChunk, n) - a);
  uint64_t* bm = bitmap + (a >> 6);
  T* rg = ring[wid];
  const int32_t tf32 = tfloor > (int64_t)INT32_MAX ? INT32_MAX : (int32_t)tfloor;
  T pre[kSplitBlk / 32];
  auto fetch = [&](uint32_t base) {
#pragma unroll
    for (uint32_t u = 0; u < kSplitBlk / 32; u++) {
      const uint32_t x = base + u * 32 + lane;
      pre[u] = x < clen ? __ldg(v + a + x) : (T)0;
    }
  };
  auto commit = [&](uint32_t base) {
#pragma unroll
    for (uint32_t u = 0; u < kSplitBlk / 32; u++) rg[(base + u * 32 + lane) & kMask] = pre[u];
  };
  fetch(0);
  commit(0);
  uint32_t filled = kSplitBlk;  // ring holds positions [filled - kRing, filled)
  fetch(filled);
  __syncwarp();
  uint32_t i = 0, j0 = 1;                          // open partition [i, j0), next candidate j0
  int64_t cmax = INT64_MIN, cmin = INT64_MAX;      // extremes of its differences (none yet)
  int ccur = 0;                                    // fast metric of [i, j0)
  uint32_t wi = 0;
  uint64_t word = 1;                               // bitmap word wi (the chunk start opens a partition)
  while (j0 < clen) {
    while (j0 + 32 > filled && filled < clen) {
      // the slot written held [filled - kRing, filled - kSplitBlk), all below j0 - 1
      __syncwarp();
      commit(filled);
      filled += kSplitBlk;
      fetch(filled);
      __syncwarp();
    }
    const uint32_t j = j0 + lane;
    const bool valid = j < clen;
    const int64_t d = valid ? (int64_t)rg[j & kMask] - (int64_t)rg[(j - 1) & kMask] : 0;
    auto cut = [&](uint32_t at) {  // position `at` opens a partition (warp-uniform)
      if ((at >> 6) != wi) {
        if (lane == 0) bm[wi] = word;
        wi = at >> 6;
        word = 0;
      }
      word |= 1ull << (at & 63u);
      cmax = INT64_MIN;
      cmin = INT64_MAX;
      ccur = 0;
      i = at;
    };
    // Whole window at once: when its differences leave the metric D of [i, j0) unchanged (D only
    // grows with the range), every candidate's C is (len + 1) D - len D = D, so the window joins
    // when D <= floor(tau S_M) and the cap allows. Differences that fit 32 bits use warp reductions
    // (and 32-bit scans below).
    const bool small = __all_sync(0xffffffffu, d >= INT32_MIN && d <= INT32_MAX);
    if (small) {
      const int32_t wmax = __reduce_max_sync(0xffffffffu, valid ? (int32_t)d : INT32_MIN);
      const int32_t wmin = __reduce_min_sync(0xffffffffu, valid ? (int32_t)d : INT32_MAX);
      const int64_t amax = cmax > (int64_t)wmax ? cmax : (int64_t)wmax;
      const int64_t amin = cmin < (int64_t)wmin ? cmin : (int64_t)wmin;
      const uint32_t jl = (clen - j0 < 32u ? clen : j0 + 32) - 1;  // the window's last candidate
      if (bitlen_u64((uint64_t)amax - (uint64_t)amin) == ccur && ccur <= tf32 && jl - i < cap) {
        cmax = amax;
        cmin = amin;
        j0 = jl + 1;
        continue;
      }
    }
    int64_t pmax = d, pmin = d;
    if (small) {
      int32_t a = (int32_t)d, b = (int32_t)d;
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const int32_t ta = __shfl_up_sync(0xffffffffu, a, o);
        const int32_t tb = __shfl_up_sync(0xffffffffu, b, o);
        if (lane >= o) {
          a = ta > a ? ta : a;
          b = tb < b ? tb : b;
        }
      }
      pmax = a;
      pmin = b;
    } else {
#pragma unroll
      for (uint32_t o = 1; o < 32; o <<= 1) {
        const int64_t tmax = __shfl_up_sync(0xffffffffu, pmax, o);
        const int64_t tmin = __shfl_up_sync(0xffffffffu, pmin, o);
        if (lane >= o) {
          pmax = tmax > pmax ? tmax : pmax;
          pmin = tmin < pmin ? tmin : pmin;
        }
      }
    }
    const int64_t nmax = cmax > pmax ? cmax : pmax, nmin = cmin < pmin ? cmin : pmin;
    const int next = bitlen_u64((uint64_t)nmax - (uint64_t)nmin);
    int cur = __shfl_up_sync(0xffffffffu, next, 1);
    if (lane == 0) cur = ccur;
    const uint32_t len = j - i;
    const int32_t C = (int32_t)(len + 1) * next - (int32_t)len * cur;
    const uint32_t rej = __ballot_sync(0xffffffffu, valid && !(len < cap && C <= tf32));
    if (rej == 0) {
      const uint32_t last = clen - 1 - j0 < 31u ? clen - 1 - j0 : 31u;
      cmax = __shfl_sync(0xffffffffu, nmax, last);
      cmin = __shfl_sync(0xffffffffu, nmin, last);
      ccur = __shfl_sync(0xffffffffu, next, last);
      j0 += 32;
    } else {
      const uint32_t at = j0 + (uint32_t)(__ffs(rej) - 1);
      cut(at);
      j0 = at + 1;
    }
  }
  if (lane == 0) bm[wi] = word;
}

// Seeded split (§3.2.2, selecting good starting positions): the greedy sweep over the count values
// u_k = v[base + dir k] (dir = +1, or -1 to read them backwards); a partition opens at u-index k when
// u_k is refused, and mark(k) records it (the first partition, at k = 0, is not marked). Same rule,
// cap and integer threshold as split_step; values are read eight ahead of the dependency chain.
template <bool NARROW, typename T, typename Mark>
__device__ __forceinline__ void sweep_dir(const T* __restrict__ v, uint64_t base, int dir, uint64_t count, uint32_t cap,
                                          int64_t tfloor, Mark mark) {
  using D = typename std::conditional<NARROW, int64_t, i128>::type;
  const int64_t step = dir;
  const T* p = v + base;
  uint64_t i = 0;
  int64_t prev = (int64_t)__ldg(p);
  D dmax = 0, dmin = 0;
  int cur = 0;
  int64_t nxt[8];
#pragma unroll
  for (int u = 0; u < 8; u++) nxt[u] = 1 + u < count ? (int64_t)__ldg(p + step * (int64_t)(1 + u)) : 0;
  for (uint64_t k0 = 1; k0 < count; k0 += 8) {
    int64_t buf[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      buf[u] = nxt[u];
      nxt[u] = k0 + 8 + u < count ? (int64_t)__ldg(p + step * (int64_t)(k0 + 8 + u)) : 0;
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint64_t k = k0 + u;
      if (k >= count) break;
      const int64_t w = buf[u];
      bool take = (k - i) < cap;
      D nmax = dmax, nmin = dmin;
      int next = 0;
      if (take) {
        const D d = (D)w - (D)prev;
        if (k == i + 1) {
          nmax = d;
          nmin = d;
        } else {
          nmax = d > nmax ? d : nmax;
          nmin = d < nmin ? d : nmin;
        }
        if (NARROW)
          next = bitlen_u64((uint64_t)nmax - (uint64_t)nmin);
        else
          next = bitlen_u128((u128)(nmax - nmin));
        const int64_t C = (int64_t)(k + 1 - i) * next - (int64_t)(k - i) * cur;
        take = C <= tfloor;
      }
      if (take) {
        cur = next;
        dmax = nmax;
        dmin = nmin;
      } else {
        mark(k);
        i = k;
        cur = 0;
        dmax = 0;
        dmin = 0;
      }
      prev = w;
    }
  }
}

// seed[c] = the first k of chunk c whose second-order delta w_{k+2} - 2 w_{k+1} + w_k has the
// shortest zigzag code (the linear regressor's smoothest window); the chunk's first position when
// it holds fewer than 3 values. A CTA per chunk; the (bits, k) minimum is reduced over the CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_chunk_seed(const T* __restrict__ v, uint64_t n, uint64_t* __restrict__ seed) {
  __shared__ uint64_t red[8];
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t a = c * kChunk, e = min(a + kChunk, n);
    uint64_t best = ~0ull;  // bits << 32 | (k - a): the minimum is the smallest bits, then the first k
    for (uint64_t k = a + threadIdx.x; k + 2 < e; k += blockDim.x) {
      const i128 d2 = (i128)(int64_t)__ldg(v + k + 2) - 2 * (i128)(int64_t)__ldg(v + k + 1) + (i128)(int64_t)__ldg(v + k);
      const u128 z = d2 >= 0 ? (u128)d2 * 2 : (u128)(-d2) * 2 - 1;
      const uint64_t key = ((uint64_t)bitlen_u128(z) << 32) | (k - a);
      best = key < best ? key : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t t = __shfl_down_sync(0xffffffffu, best, o);
      best = t < best ? t : best;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < 8; w++) best = red[w] < best ? red[w] : best;
      seed[c] = best == ~0ull ? a : a + (best & 0xFFFFFFFFull);
    }
    __syncthreads();
  }
}

// cls[c] for chunk c (a CTA per chunk): kChunkNarrow when every value lies in (-2^62, 2^62) as
// int64; kChunkLanes when the chunk goes to the one-lane-per-chunk sweep: values beyond that range,
// or cuts expected densely. A two-value partition [i, i + 2) refuses v_{i+2} exactly when
// 3 bitlen(|second difference|) > floor(tau S_M) (C = 3 D - 2 * 0), so the share of positions with
// such a second difference estimates how many partitions stay that short; above 1 in 12 in any of
// the sampled windows (the chunk's slowest part sets its sweep time) the per-lane sweep (about one
// dependent step per position) beats the warp's (one step per partition). The class changes only
// the speed.
template <typename T>
__global__ void k_chunk_class(const T* __restrict__ v, uint64_t n, int64_t tfloor, uint8_t* __restrict__ cls) {
  constexpr uint32_t kWin = kClassSample / kClassWindows;  // positions per sampled window
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  const int64_t lim = (int64_t)1 << 62;
  __shared__ unsigned int sharp[kClassWindows];
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t a = c * kChunk, e = min(a + kChunk, n);
    if (threadIdx.x < kClassWindows) sharp[threadIdx.x] = 0;
    __syncthreads();
    int bad = 0;
    if (sizeof(T) == 8)
      for (uint64_t j = a + threadIdx.x; j < e; j += blockDim.x) {
        const int64_t w = (int64_t)__ldg(v + j);
        bad |= (w <= -lim || w >= lim) ? 1 : 0;
      }
    // kClassWindows windows of kWin positions spread evenly over the chunk (a warp's 32 positions
    // fall in one window); wrapping arithmetic: an estimate only
    for (uint32_t k = threadIdx.x; k < kClassSample; k += blockDim.x) {
      const uint32_t s = k / kWin;
      const uint64_t j = a + (uint64_t)s * (kChunk / kClassWindows) + (k % kWin);
      bool sh = false;
      if (j > a && j + 1 < e) {
        const uint64_t d2 = (uint64_t)(int64_t)__ldg(v + j + 1) - 2 * (uint64_t)(int64_t)__ldg(v + j) +
                            (uint64_t)(int64_t)__ldg(v + j - 1);
        const uint64_t mag = (int64_t)d2 < 0 ? 0 - d2 : d2;
        sh = 3 * (int64_t)bitlen_u64(mag) > tfloor;
      }
      const unsigned int cnt = __popc(__ballot_sync(0xffffffffu, sh));
      if ((threadIdx.x & 31u) == 0 && cnt) atomicAdd(&sharp[s], cnt);
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
      bool lanes = bad != 0;
      for (uint32_t s = 0; s < kClassWindows; s++) {
        const uint64_t w0 = a + (uint64_t)s * (kChunk / kClassWindows);
        const uint64_t wl = w0 < e ? min((uint64_t)kWin, e - w0) : 0;
        lanes = lanes || 12ull * sharp[s] > wl;
      }
      cls[c] = (uint8_t)((bad ? 0 : kChunkNarrow) | (lanes ? kChunkLanes : 0));
    }
    __syncthreads();  // sharp is reset for the next chunk
  }
}

// one chunk of the seeded split: partitions grow from the chunk's seed to the right, and to the
// left by the same sweep over the values read backwards (a partition refused there at u-index k
// starts at seed - k); the chunk edge and the seed are cuts. The thread owns the chunk's words.
template <bool NARROW, typename T>
__device__ __forceinline__ void split_chunk_seeded(const T* __restrict__ v, uint64_t a, uint64_t e, uint64_t seed,
                                                   uint32_t cap, int64_t tfloor, uint64_t* __restrict__ bitmap) {
  for (uint64_t w = a >> 6; w <= ((e - 1) >> 6); w++) bitmap[w] = 0;
  auto set = [&](uint64_t pos) { bitmap[pos >> 6] |= 1ull << (pos & 63); };
  set(a);
  set(seed);
  if (seed > a) sweep_dir<NARROW>(v, seed - 1, -1, seed - a, cap, tfloor, [&](uint64_t k) { set(seed - k); });
  sweep_dir<NARROW>(v, seed, 1, e - seed, cap, tfloor, [&](uint64_t k) { set(seed + k); });
}


// the seeded split: chunk c's partitions grow from seeds[c] (k_chunk_seed) both ways; a thread per chunk
template <typename T>
__global__ void k_split_seeded(const T* __restrict__ values, uint64_t n, uint32_t cap, int64_t tfloor,
                               const uint8_t* __restrict__ cls, const uint64_t* __restrict__ seeds,
                               uint64_t* __restrict__ bitmap) {
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = c * kChunk;
    const uint64_t e = min(a + kChunk, n);
    if (cls[c] & kChunkNarrow)
      split_chunk_seeded<true>(values, a, e, seeds[c], cap, tfloor, bitmap);
    else
      split_chunk_seeded<false>(values, a, e, seeds[c], cap, tfloor, bitmap);
  }
}


__global__ void k_popc(const uint64_t* __restrict__ bitmap, uint64_t nw, uint64_t* __restrict__ cnt) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nw;
       w += (uint64_t)gridDim.x * blockDim.x)
    cnt[w] = (uint64_t)__popcll(bitmap[w]);
}

__global__ void k_scatter_starts(const uint64_t* __restrict__ bitmap, uint64_t nw,
                                 const uint64_t* __restrict__ pos, uint64_t n, uint64_t m,
                                 uint64_t* __restrict__ starts) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nw;
       w += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t bits = bitmap[w];
    uint64_t k = pos[w];
    while (bits) {
      const int t = __ffsll((long long)bits) - 1;
      starts[k++] = w * 64 + (uint64_t)t;
      bits &= bits - 1;
    }
    if (w == 0) starts[m] = n;
  }
}

// Fixed-partition size search (§3.2.1): total S_M + len * b over partitions of L values cut from
// each of k sampled subsequences of N values (starts[s]), the last of each possibly short.
// Thread per partition for L <= kTinySpan, warp per partition above; one atomic per warp.
__global__ void k_sample_sizes_thread(const void* __restrict__ values, int dtype, const uint64_t* __restrict__ starts,
                                      uint64_t k, uint32_t N, uint32_t L, int model,
                                      unsigned long long* __restrict__ total) {
  const uint64_t P = (N + L - 1) / L, count = k * P;
  uint64_t acc = 0;
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < count; t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = t / P, j = t - s * P;
    const uint32_t len = (uint32_t)min((uint64_t)L, (uint64_t)N - j * L);
    const FitResult R = fit_range<1>(values, dtype, starts[s] + j * L, len, model, 0, nullptr);
    acc += kSmBits + (uint64_t)len * R.b;
  }
  acc = warp_sum_u64(acc);
  if ((threadIdx.x & 31u) == 0 && acc) atomicAdd(total, (unsigned long long)acc);
}

__global__ void k_sample_sizes_warp(const void* __restrict__ values, int dtype, const uint64_t* __restrict__ starts,
                                    uint64_t k, uint32_t N, uint32_t L, int model,
                                    unsigned long long* __restrict__ total) {
  const uint64_t P = (N + L - 1) / L, count = k * P;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint64_t acc = 0;
  for (uint64_t t = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; t < count; t += nw) {
    const uint64_t s = t / P, j = t - s * P;
    const uint32_t len = (uint32_t)min((uint64_t)L, (uint64_t)N - j * L);
    const FitResult R = fit_range<32>(values, dtype, starts[s] + j * L, len, model, lane, nullptr);
    acc += kSmBits + (uint64_t)len * R.b;
  }
  if (lane == 0 && acc) atomicAdd(total, (unsigned long long)acc);
}

int grid_for(uint64_t items, int per_block, int max_blocks_per_sm) {
  const uint64_t need = (items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)sm_count() * max_blocks_per_sm;
  return (int)(need < cap ? (need ? need : 1) : cap);
}

// ----------------------------------------------------------------------------------------- merge
//
// The moments of a span's values (w = the value as two's complement int64, x = the local index):
// T0 = sum w, T1 = sum x w, and min and max of w. Two adjacent spans' moments combine exactly (the
// right span's x shifts by the left span's length: T1 gains N_left T0_right), and they give the
// least-squares moment S = sum (2x - (N-1)) w = 2 T1 - (N-1) T0 of the fit and its bounds, so a
// refit needs one pass over the values: the residual range under the snapped line (none for the
// constant model, whose residuals are the values themselves). The moments move with the partitions
// when a round compacts them (a merged pair's are combined then), and the final partitions' fits
// are taken once, from their moments, at the end.
// a pair too long for one warp: its residual range is reduced over pieces of kPiece values
struct LongPair {
  uint64_t j;  // pair index
  uint64_t k;  // slot of its left partition
  uint64_t a;  // first position
  FitParams P;
  uint32_t N;
  uint32_t pad;
};

constexpr uint32_t kTinySpan = 256;    // size search: a thread per sampled partition up to this size
constexpr uint32_t kWarpSpan = 4096;   // a warp fits longer pairs up to this long (split partitions: any)
constexpr uint32_t kPiece = 2048;      // values per piece of a longer pair
constexpr int kGroupBlock = 256;       // 8 warps, each taking 32 spans at a time
constexpr uint32_t kStageBytes = 4096; // per warp: a group's values are staged when they fit

struct MergeWork {
  LongPair* longs;
  uint64_t* pieces;
  unsigned long long* counters;  // [long pairs, pieces]
  long long* lo;                 // per long pair
  long long* hi;
  unsigned long long* zmax;
};

// Full fits of spans. MODE 1: every partition of the split (its moments from a pass over its
// values, into stats[j]; size S_M + len * b into size_out[j]). MODE 2: the dirty adjacent pairs
// [st[j], st[j + 2)) (moments combined from stats[j] and stats[j + 1]; merged size into
// size_out[j]). MODE 3: the final partitions (moments stats[j]; record into rec[j], as the
// encoder's fit writes it). A warp takes 32 consecutive spans; when their values cover at most
// kStageBytes it first stages them in shared memory with coalesced loads. A lane then fits its own
// span when it is at most kLaneSpan long, tiles of eight lanes fit spans up to kTileSpan, the warp
// fits longer ones together, and spans longer than
// kWarpSpan (modes 2 and 3, not staged) go to the piece list, where many warps share their residual
// pass (k_pair_pieces, then k_pair_finish).
template <typename T, int MODE>
__global__ void __launch_bounds__(kGroupBlock, 3)
    k_span_groups(const T* __restrict__ v, const uint64_t* __restrict__ st, uint64_t count, uint32_t cap, int model,
                  const uint8_t* __restrict__ dirty, SpanStats* __restrict__ stats, uint64_t* __restrict__ size_out,
                  Record* __restrict__ rec, MergeWork mw) {
  constexpr int W = MODE == 2 ? 2 : 1;
  __shared__ __align__(16) unsigned char stage_raw[kGroupBlock / 32][kStageBytes];
  constexpr uint64_t kStageVals = kStageBytes / sizeof(T);
  const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
  T* stage = reinterpret_cast<T*>(stage_raw[wib]);
  const uint64_t ngroups = (count + 31) / 32;
  const uint64_t gw = (uint64_t)gridDim.x * (kGroupBlock / 32);
  for (uint64_t g = (uint64_t)blockIdx.x * (kGroupBlock / 32) + wib; g < ngroups; g += gw) {
    const uint64_t j = g * 32 + lane;
    bool act = j < count && (MODE != 2 || dirty[j]);
    if (!__any_sync(kFull, act)) continue;
    uint64_t a = 0, c = 0;
    if (act) {
      a = st[j];
      c = st[j + W];
      if (W == 2 && c - a > cap) {  // pairs beyond the cap never merge
        size_out[j] = kNone;
        act = false;
      }
    }
    const uint32_t N = act ? (uint32_t)(c - a) : 0u;
    const uint64_t ga = xw_min_u(act ? a : ~0ull), gc = xw_max_u(act ? c : 0ull);
    const bool staged = ga != ~0ull && gc - ga <= kStageVals;
    if (staged) {
      for (uint64_t t = lane; t < gc - ga; t += 32) stage[t] = __ldg(v + ga + t);
      __syncwarp();
    }
    const T* src = staged ? stage + (a - ga) : v + a;
    // moments
    SpanStats S;
    S.T0 = S.T1 = 0;
    S.mn = S.mx = 0;
    if (MODE == 1) {
      if (act && N <= kLaneSpan) S = stats_part(src, 0, N, 1);
      coop_stats<8>(__ballot_sync(kFull, act && N > kLaneSpan && N <= kTileSpan), src, N, S);
      coop_stats<32>(__ballot_sync(kFull, act && N > kTileSpan), src, N, S);
    } else if (MODE == 2 && act) {
      S = combine_stats(stats[j], st[j + 1] - a, stats[j + 1]);
    } else if (act) {
      S = stats[j];
    }
    // parameters (fit.cuh steps 1-3)
    const bool lin = model == LECO_MODEL_LINEAR && N >= 2;
    FitParams P;
    P.B = 0;
    P.fb_shift = 0;
    P.s = 0;
    P.fallback = 0;
    if (act) P = solve_params(lin ? 2 * S.T1 - mul_i128_u64(S.T0, N - 1) : (i128)0, S.mx, S.mn, N, lin);
    // residual range (step 4)
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    uint64_t zmax = 0;
    const bool need = act && (lin || P.fallback);
    if (act && !need) {  // constant model on its grid: the residuals are the values
      lo = S.mn;
      hi = S.mx;
    }
    const bool by_lane = need && N <= kLaneSpan;
    const bool by_warp = need && N > kLaneSpan && (MODE == 1 || staged || N <= kWarpSpan);
    const bool by_pieces = need && !by_lane && !by_warp;
    if (by_lane) resid_part(src, 0, N, 1, P, lo, hi, zmax);
    coop_resid<8>(__ballot_sync(kFull, by_warp && N <= kTileSpan), src, N, P, lo, hi, zmax);
    coop_resid<32>(__ballot_sync(kFull, by_warp && N > kTileSpan), src, N, P, lo, hi, zmax);
    if (by_pieces) {
      const uint32_t np = (N + kPiece - 1) / kPiece;
      const unsigned long long li = atomicAdd(&mw.counters[0], 1ull);
      const unsigned long long pb = atomicAdd(&mw.counters[1], (unsigned long long)np);
      LongPair lp;
      lp.j = j;
      lp.k = 0;
      lp.a = a;
      lp.P = P;
      lp.N = N;
      lp.pad = 0;
      mw.longs[li] = lp;
      mw.lo[li] = INT64_MAX;
      mw.hi[li] = INT64_MIN;
      mw.zmax[li] = 0;
      for (uint32_t q = 0; q < np; q++) mw.pieces[pb + q] = ((uint64_t)li << 16) | q;
    }
    if (act && !by_pieces) {  // steps 5-6
      if (MODE == 3) {
        const FitResult R = finish_fit(P, lo, hi, zmax);
        Record r;
        r.theta0 = R.theta0;
        r.theta1 = R.theta1;
        r.start = a;
        r.word3 = make_w3(0, R.b, R.s, 1);
        rec[j] = r;
      } else {
        size_out[j] = kSmBits + (uint64_t)N * finish_width(P, lo, hi, zmax);
      }
      if (MODE == 1) stats[j] = S;
    }
    __syncwarp();  // the stage is reused by the next group
  }
}

// residual range of one piece of a long pair per warp, folded into the pair's range by atomics
template <typename T>
__global__ void __launch_bounds__(256) k_pair_pieces(const T* __restrict__ v, MergeWork mw) {
  const uint64_t np = *(volatile unsigned long long*)&mw.counters[1];
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t pi = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; pi < np; pi += nw) {
    const uint64_t e = mw.pieces[pi];
    const uint64_t li = e >> 16;
    const uint32_t q = (uint32_t)(e & 0xFFFFu);
    const LongPair L = mw.longs[li];
    const uint32_t x0 = q * kPiece, x1 = min(x0 + kPiece, L.N);
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    uint64_t z = 0;
    resid_part(v + L.a, x0 + lane, x1, 32, L.P, lo, hi, z);
    lo = warp_min_i64(lo);
    hi = warp_max_i64(hi);
    z = warp_max_u64(z);
    if (lane == 0) {
      atomicMin(&mw.lo[li], (long long)lo);
      atomicMax(&mw.hi[li], (long long)hi);
      atomicMax(&mw.zmax[li], (unsigned long long)z);
    }
  }
}

// steps 5-6 of the long spans: their merged size (msz) or their record (rec)
__global__ void k_pair_finish(MergeWork mw, uint64_t* __restrict__ msz, Record* __restrict__ rec) {
  const uint64_t nl = *(volatile unsigned long long*)&mw.counters[0];
  for (uint64_t li = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x) {
    const LongPair L = mw.longs[li];
    if (rec) {
      const FitResult R = finish_fit(L.P, (int64_t)mw.lo[li], (int64_t)mw.hi[li], (uint64_t)mw.zmax[li]);
      Record r;
      r.theta0 = R.theta0;
      r.theta1 = R.theta1;
      r.start = L.a;
      r.word3 = make_w3(0, R.b, R.s, 1);
      rec[L.j] = r;
    } else {
      msz[L.j] = kSmBits + (uint64_t)L.N * finish_width(L.P, (int64_t)mw.lo[li], (int64_t)mw.hi[li], (uint64_t)mw.zmax[li]);
    }
  }
}

__device__ __forceinline__ bool pair_gain(const uint64_t* sz, const uint64_t* msz, uint64_t j, int64_t* g) {
  if (msz[j] == kNone) return false;
  *g = (int64_t)(sz[j] + sz[j + 1]) - (int64_t)msz[j];
  return true;
}

// priority order of two pairs: gain, then the hash of the start, then the smaller start
__device__ __forceinline__ bool beats(int64_t g1, uint64_t s1, int64_t g2, uint64_t s2) {
  if (g1 != g2) return g1 > g2;
  const uint64_t h1 = splitmix64(s1), h2 = splitmix64(s2);
  if (h1 != h2) return h1 > h2;
  return s1 < s2;
}

// sel[j]: pair j merges this round; keep[p]: partition p survives (it was not merged into its left
// neighbour); *nsel counts the merging pairs
__global__ void k_select(const uint64_t* __restrict__ st, const uint64_t* __restrict__ sz,
                         const uint64_t* __restrict__ msz, uint64_t m, uint8_t* __restrict__ sel,
                         uint64_t* __restrict__ keep, unsigned long long* __restrict__ nsel) {
  uint32_t local = 0;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
    bool ok = false;
    if (j + 1 < m) {
      int64_t g;
      ok = pair_gain(sz, msz, j, &g) && g > 0;
      if (ok && j > 0) {
        int64_t gl;
        if (pair_gain(sz, msz, j - 1, &gl) && !beats(g, st[j], gl, st[j - 1])) ok = false;
      }
      if (ok && j + 2 < m) {
        int64_t gr;
        if (pair_gain(sz, msz, j + 1, &gr) && !beats(g, st[j], gr, st[j + 1])) ok = false;
      }
    }
    sel[j] = ok ? 1 : 0;
    local += ok ? 1u : 0u;
    // partition j + 1 is absorbed when pair j merges; partition 0 always survives
    if (j + 1 < m) keep[j + 1] = ok ? 0ull : 1ull;
    if (j == 0) keep[0] = 1ull;
  }
  local = (uint32_t)warp_sum_u64(local);
  if ((threadIdx.x & 31u) == 0 && local) atomicAdd(nsel, (unsigned long long)local);
}

// the next round's arrays; a merged pair's moments are combined. Every load a partition needs is
// issued before the first branch, so the loads of one thread overlap.
__global__ void k_compact(const uint64_t* __restrict__ st, const uint64_t* __restrict__ sz,
                          const uint64_t* __restrict__ msz, const uint8_t* __restrict__ sel,
                          const uint64_t* __restrict__ newidx, const SpanStats* __restrict__ stats, uint64_t m,
                          uint64_t n, uint64_t new_m, uint64_t* __restrict__ nst, uint64_t* __restrict__ nsz,
                          uint64_t* __restrict__ nmsz, uint8_t* __restrict__ ndirty, SpanStats* __restrict__ nstats) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const bool absorbed = p > 0 && sel[p - 1];  // merged into p - 1
    const bool mp = p + 1 < m && sel[p];
    const bool mq2 = p + 3 < m && sel[p + 2];  // the next survivor's pair when p merges
    const bool mq1 = p + 2 < m && sel[p + 1];  // ... when it does not
    const uint64_t k = newidx[p];
    const uint64_t s0 = st[p];
    const uint64_t szp = sz[p];
    const uint64_t mszp = p + 1 < m ? msz[p] : 0;
    const uint64_t s1 = p + 1 < m ? st[p + 1] : n;
    if (absorbed) continue;
    const SpanStats sp = stats[p];
    nst[k] = s0;
    nsz[k] = mp ? mszp : szp;
    nstats[k] = mp ? combine_stats(sp, s1 - s0, stats[p + 1]) : sp;
    const uint64_t q = mp ? p + 2 : p + 1;  // next surviving partition
    if (q < m) {
      const bool d = mp || (mp ? mq2 : mq1);
      ndirty[k] = d ? 1 : 0;
      if (!d) nmsz[k] = mszp;
    }
    if (k == 0) nst[new_m] = n;
  }
}



template <typename T>
cudaError_t dalloc(T** p, uint64_t elems, cudaStream_t st) {
  return dev_alloc((void**)p, (elems ? elems : 1) * sizeof(T), st);
}

int group_grid(uint64_t count) {
  const uint64_t groups = (count + 31) / 32;
  return grid_for((groups + kGroupBlock / 32 - 1) / (kGroupBlock / 32), 1, 3);
}

// one mode of k_span_groups over count spans, then (modes 2 and 3) the pieces of the long ones
template <typename T>
cudaError_t span_groups(const void* values, int mode, const uint64_t* st, uint64_t count, uint32_t cap, int model,
                        const uint8_t* dirty, SpanStats* stats, uint64_t* size_out, Record* rec, const MergeWork& mw,
                        cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const T* v = static_cast<const T*>(values);
  if (mode != 1) {
    const cudaError_t e = cudaMemsetAsync(mw.counters, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  if (mode == 1)
    k_span_groups<T, 1><<<group_grid(count), kGroupBlock, 0, s>>>(v, st, count, cap, model, dirty, stats, size_out,
                                                                  rec, mw);
  else if (mode == 2)
    k_span_groups<T, 2><<<group_grid(count), kGroupBlock, 0, s>>>(v, st, count, cap, model, dirty, stats, size_out,
                                                                  rec, mw);
  else
    k_span_groups<T, 3><<<group_grid(count), kGroupBlock, 0, s>>>(v, st, count, cap, model, dirty, stats, size_out,
                                                                  rec, mw);
  if (mode != 1) {
    k_pair_pieces<T><<<sm_count() * 8, 256, 0, s>>>(v, mw);
    k_pair_finish<<<sm_count() * 2, 256, 0, s>>>(mw, size_out, mode == 3 ? rec : nullptr);
  }
  return cudaGetLastError();
}

}  // namespace


// Fixed partition-size search (§3.2.1), in the reading the oracle states (R9): SplitMix64-placed
// sample subsequences, an exponential phase over powers of two that ends after the first size above
// its predecessor's, then a back search with halving steps, stopping when a move gains < 0.01 %.
cudaError_t search_partition_size(const void* values, int dtype, uint64_t n, int model, uint32_t N, double frac,
                                  uint64_t seed, uint32_t* best_L, uint64_t* best_bits, uint64_t* evals,
                                  cudaStream_t st) {
  *best_L = 1;
  *best_bits = 0;
  *evals = 0;
  if (n == 0) return cudaSuccess;
  if (n < N) N = (uint32_t)n;
  std::vector<uint64_t> h_starts;
  if (n <= N) {
    h_starts.push_back(0);
  } else {
    uint64_t k = (uint64_t)(frac * (double)n / (double)N);
    if (k < 1) k = 1;
    for (uint64_t i = 0; i < k; i++) h_starts.push_back(splitmix64(seed + i) % (n - N + 1));
  }
  const uint64_t k = h_starts.size();
  uint64_t* d_starts = nullptr;
  unsigned long long* d_total = nullptr;
  cudaError_t e = dalloc(&d_starts, k, st);
  if (e == cudaSuccess) e = dalloc(&d_total, 1, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_starts, h_starts.data(), 8 * k, cudaMemcpyHostToDevice, st);
  std::map<uint32_t, uint64_t> cache;
  auto size_at = [&](uint32_t L) -> uint64_t {
    auto it = cache.find(L);
    if (it != cache.end()) return it->second;
    unsigned long long total = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(d_total, 0, 8, st);
    const uint64_t parts = k * ((N + L - 1) / L);
    if (e == cudaSuccess) {
      if (L <= kTinySpan)
        k_sample_sizes_thread<<<grid_for(parts, 256, 8), 256, 0, st>>>(values, dtype, d_starts, k, N, L, model, d_total);
      else
        k_sample_sizes_warp<<<grid_for(parts * 32, 256, 8), 256, 0, st>>>(values, dtype, d_starts, k, N, L, model,
                                                                          d_total);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, d_total, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cache[L] = total;
    return total;
  };
  uint32_t best = 1;
  uint64_t best_s = size_at(1), prev_s = best_s;
  for (uint64_t L = 2; e == cudaSuccess; L *= 2) {  // exponential phase
    const uint32_t LL = (uint32_t)(L < N ? L : N);
    const uint64_t s = size_at(LL);
    if (s < best_s) {
      best_s = s;
      best = LL;
    }
    if (s > prev_s || LL == N) break;
    prev_s = s;
  }
  for (uint32_t step = best / 2; step > 0 && e == cudaSuccess;) {  // back search
    uint32_t cand = best;
    uint64_t cand_s = best_s;
    if (best > step) {
      const uint64_t s = size_at(best - step);
      if (s < cand_s) {
        cand_s = s;
        cand = best - step;
      }
    }
    if (best + step <= N) {
      const uint64_t s = size_at(best + step);
      if (s < cand_s) {
        cand_s = s;
        cand = best + step;
      }
    }
    if (cand == best) {
      step /= 2;
      continue;
    }
    const bool small_gain = (best_s - cand_s) * 10000 < best_s;
    best = cand;
    best_s = cand_s;
    if (small_gain) break;
  }
  if (d_starts) cudaFreeAsync(d_starts, st);
  if (d_total) cudaFreeAsync(d_total, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) {
    *best_L = best;
    *best_bits = best_s;
    *evals = cache.size();
  }
  return e;
}

// Runs split + merge; writes m+1 starts to starts_out (capacity n+1) and m to *m_out. rec_out:
// when non-null, receives m records (a new device allocation from the library pool; the caller
// frees it) holding the full fit of every final partition, as the encoder's fit writes them.
cudaError_t var_partition_fit(const void* values, int dtype, uint64_t n, double tau, uint32_t cap, int model,
                              bool seeded, uint64_t* starts_out, uint64_t* m_out, Record** rec_out, cudaStream_t st) {
  *m_out = 0;
  if (rec_out) *rec_out = nullptr;
  if (n == 0) {
    const uint64_t zero = 0;
    cudaError_t e = cudaMemcpyAsync(starts_out, &zero, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  const bool u32 = dtype == LECO_U32;
  const double thresh = tau * (double)kSmBits;
  const uint64_t nw = (n + 63) / 64;
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  // C <= tau * S_M for an integer C: C <= floor(tau * S_M) (thresh >= 0, below 2^62 here)
  const int64_t tfloor = thresh < 4.0e18 ? (int64_t)floor(thresh) : INT64_MAX;
  uint64_t m = 0;
  cudaError_t e = cudaSuccess;
  {  // split
    uint64_t *bitmap = nullptr, *cnt = nullptr, *pos = nullptr, *scan_scratch = nullptr, *d_total = nullptr;
    uint64_t* seeds = nullptr;
    const uint64_t scan_elems = nw / 2048 + 2;
    if (e == cudaSuccess) e = dalloc(&bitmap, nw, st);
    if (e == cudaSuccess) e = dalloc(&cnt, nw, st);
    if (e == cudaSuccess) e = dalloc(&pos, nw, st);
    if (e == cudaSuccess) e = dalloc(&scan_scratch, scan_elems + 1, st);
    if (e == cudaSuccess) e = dalloc(&d_total, 1, st);
    if (e == cudaSuccess && seeded) e = dalloc(&seeds, nchunks, st);
    uint8_t* cls = reinterpret_cast<uint8_t*>(cnt);  // chunk classes; cnt is not used until the popcount
    if (e == cudaSuccess) {
      const int wgrid = (int)((nchunks + kSplitWarps - 1) / kSplitWarps);
      if (u32) {
        const uint32_t* v = static_cast<const uint32_t*>(values);
        k_chunk_class<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(v, n, tfloor, cls);
        if (seeded) {
          k_chunk_seed<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(v, n, seeds);
          k_split_seeded<<<grid_for(nchunks, 32, 32), 32, 0, st>>>(v, n, cap, tfloor, cls, seeds, bitmap);
        } else {
          e = cudaMemsetAsync(bitmap, 0, 8 * nw, st);
          if (e == cudaSuccess) {
            k_split_lanes<<<(int)((nchunks + 31) / 32), 32, 0, st>>>(v, n, cap, tfloor, cls, bitmap);
            k_split_warp<<<wgrid, 32 * kSplitWarps, 0, st>>>(v, n, cap, tfloor, cls, bitmap);
          }
        }
      } else {
        const uint64_t* v = static_cast<const uint64_t*>(values);
        k_chunk_class<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(v, n, tfloor, cls);
        if (seeded) {
          k_chunk_seed<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(v, n, seeds);
          k_split_seeded<<<grid_for(nchunks, 32, 32), 32, 0, st>>>(v, n, cap, tfloor, cls, seeds, bitmap);
        } else {
          e = cudaMemsetAsync(bitmap, 0, 8 * nw, st);
          if (e == cudaSuccess) {
            k_split_lanes<<<(int)((nchunks + 31) / 32), 32, 0, st>>>(v, n, cap, tfloor, cls, bitmap);
            k_split_warp<<<wgrid, 32 * kSplitWarps, 0, st>>>(v, n, cap, tfloor, cls, bitmap);
          }
        }
      }
      if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_popc<<<grid_for(nw, 256, 8), 256, 0, st>>>(bitmap, nw, cnt);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_u64(cnt, nw, pos, scan_scratch, d_total, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&m, d_total, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      k_scatter_starts<<<grid_for(nw, 256, 8), 256, 0, st>>>(bitmap, nw, pos, n, m, starts_out);
      e = cudaGetLastError();
    }
    for (uint64_t* p : {bitmap, cnt, pos, scan_scratch, d_total, seeds})
      if (p) cudaFreeAsync(p, st);
  }
  if (e != cudaSuccess) return e;

  // merge state
  const uint64_t m0 = m;
  SpanStats *stats = nullptr, *stats_b = nullptr;
  uint64_t *st_b = nullptr, *sz_a = nullptr, *sz_b = nullptr;
  uint64_t *msz_a = nullptr, *msz_b = nullptr, *keep = nullptr, *newidx = nullptr, *scr = nullptr, *d_total = nullptr;
  uint8_t *dirty_a = nullptr, *dirty_b = nullptr, *sel = nullptr;
  unsigned long long* d_nsel = nullptr;
  MergeWork mw;
  mw.longs = nullptr;
  mw.pieces = nullptr;
  mw.counters = nullptr;
  mw.lo = nullptr;
  mw.hi = nullptr;
  mw.zmax = nullptr;
  const uint64_t long_cap = 2 * n / kWarpSpan + 2;
  const uint64_t piece_cap = 2 * n / kPiece + long_cap + 2;
  const uint64_t scr_elems = m0 / 2048 + 2;
  if (e == cudaSuccess) e = dalloc(&stats, m0, st);
  if (e == cudaSuccess) e = dalloc(&stats_b, m0, st);
  if (e == cudaSuccess) e = dalloc(&st_b, m0 + 1, st);
  if (e == cudaSuccess) e = dalloc(&sz_a, m0, st);
  if (e == cudaSuccess) e = dalloc(&sz_b, m0, st);
  if (e == cudaSuccess) e = dalloc(&msz_a, m0, st);
  if (e == cudaSuccess) e = dalloc(&msz_b, m0, st);
  if (e == cudaSuccess) e = dalloc(&keep, m0, st);
  if (e == cudaSuccess) e = dalloc(&newidx, m0, st);
  if (e == cudaSuccess) e = dalloc(&scr, scr_elems + 1, st);
  if (e == cudaSuccess) e = dalloc(&d_total, 1, st);
  if (e == cudaSuccess) e = dalloc(&dirty_a, m0, st);
  if (e == cudaSuccess) e = dalloc(&dirty_b, m0, st);
  if (e == cudaSuccess) e = dalloc(&sel, m0, st);
  if (e == cudaSuccess) e = dalloc(&d_nsel, 1, st);
  if (e == cudaSuccess) e = dalloc(&mw.longs, long_cap, st);
  if (e == cudaSuccess) e = dalloc(&mw.pieces, piece_cap, st);
  if (e == cudaSuccess) e = dalloc(&mw.counters, 2, st);
  if (e == cudaSuccess) e = dalloc(&mw.lo, long_cap, st);
  if (e == cudaSuccess) e = dalloc(&mw.hi, long_cap, st);
  if (e == cudaSuccess) e = dalloc(&mw.zmax, long_cap, st);
  uint64_t* cur_st = starts_out;
  uint64_t* nxt_st = st_b;
  // every split partition's moments, fit and size
  if (e == cudaSuccess)
    e = u32 ? span_groups<uint32_t>(values, 1, cur_st, m, cap, model, nullptr, stats, sz_a, nullptr, mw, st)
            : span_groups<uint64_t>(values, 1, cur_st, m, cap, model, nullptr, stats, sz_a, nullptr, mw, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dirty_a, 1, m, st);
  while (e == cudaSuccess && m > 1) {
    e = u32 ? span_groups<uint32_t>(values, 2, cur_st, m - 1, cap, model, dirty_a, stats, msz_a, nullptr, mw, st)
            : span_groups<uint64_t>(values, 2, cur_st, m - 1, cap, model, dirty_a, stats, msz_a, nullptr, mw, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_nsel, 0, 8, st);
    if (e != cudaSuccess) break;
    k_select<<<grid_for(m, 256, 8), 256, 0, st>>>(cur_st, sz_a, msz_a, m, sel, keep, d_nsel);
    unsigned long long nsel = 0;
    e = cudaMemcpyAsync(&nsel, d_nsel, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || nsel == 0) break;
    e = scan_u64(keep, m, newidx, scr, d_total, st);
    if (e != cudaSuccess) break;
    const uint64_t new_m = m - nsel;
    k_compact<<<grid_for(m, 256, 8), 256, 0, st>>>(cur_st, sz_a, msz_a, sel, newidx, stats, m, n, new_m, nxt_st,
                                                   sz_b, msz_b, dirty_b, stats_b);
    e = cudaGetLastError();
    std::swap(cur_st, nxt_st);
    std::swap(sz_a, sz_b);
    std::swap(msz_a, msz_b);
    std::swap(dirty_a, dirty_b);
    std::swap(stats, stats_b);
    m = new_m;
  }
  if (e == cudaSuccess && rec_out) {
    e = dalloc(rec_out, m, st);  // the final partitions' fits from their moments
    if (e == cudaSuccess)
      e = u32 ? span_groups<uint32_t>(values, 3, cur_st, m, cap, model, nullptr, stats, nullptr, *rec_out, mw, st)
              : span_groups<uint64_t>(values, 3, cur_st, m, cap, model, nullptr, stats, nullptr, *rec_out, mw, st);
  }
  if (e == cudaSuccess && cur_st != starts_out)
    e = cudaMemcpyAsync(starts_out, cur_st, (m + 1) * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(cur_st == starts_out ? nxt_st : cur_st, st);  // st_b, wherever it ended up
  for (void* p : {(void*)stats, (void*)stats_b, (void*)sz_a,
                  (void*)sz_b, (void*)msz_a, (void*)msz_b, (void*)keep, (void*)newidx, (void*)scr, (void*)d_total,
                  (void*)dirty_a, (void*)dirty_b, (void*)sel, (void*)d_nsel, (void*)mw.longs, (void*)mw.pieces,
                  (void*)mw.counters, (void*)mw.lo, (void*)mw.hi, (void*)mw.zmax})
    if (p) cudaFreeAsync(p, st);
  if (e != cudaSuccess && rec_out && *rec_out) {
    cudaFreeAsync(*rec_out, st);
    *rec_out = nullptr;
  }
  if (e == cudaSuccess) *m_out = m;
  return e;
}

cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap, int model, bool seeded,
                          uint64_t* starts_out, uint64_t* m_out, cudaStream_t st) {
  return var_partition_fit(values, dtype, n, tau, cap, model, seeded, starts_out, m_out, nullptr, st);
}

cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap,
                          int model, uint64_t* starts_out, uint64_t* m_out, cudaStream_t st) {
  return var_partition_fit(values, dtype, n, tau, cap, model, false, starts_out, m_out, nullptr, st);
}

namespace {
// lenbits[p] = len_p * b_p and the widest b, from records whose fits are done (variable partitions)
__global__ void k_lenbits(const Record* __restrict__ rec, const uint64_t* __restrict__ starts, uint64_t m,
                          uint64_t* __restrict__ lenbits, uint32_t* __restrict__ max_b) {
  uint32_t mb = 0;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = w3_b(rec[p].word3);
    lenbits[p] = (starts[p + 1] - starts[p]) * b;
    mb = max(mb, b);
  }
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_down_sync(kFull, mb, o));
  if ((threadIdx.x & 31u) == 0 && mb) atomicMax(max_b, mb);
}
}  // namespace

cudaError_t launch_lenbits(const Record* rec, const uint64_t* starts, uint64_t m, uint64_t* lenbits, uint32_t* max_b,
                           cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(max_b, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess || m == 0) return e;
  k_lenbits<<<grid_for(m, 256, 8), 256, 0, st>>>(rec, starts, m, lenbits, max_b);
  return cudaGetLastError();
}

}  // namespace leco

