// Variable-length partitioning on the GPU (§3.2.2): split, then merge.
//
// Split: the sequence is cut into chunks of kChunk values (chunk edges always start a partition);
// inside a chunk one thread grows partitions left to right: v_j joins the open partition [i, j)
// iff C = (j+1-i) D(v[i,j+1)) - (j-i) D(v[i,j)) <= tau * S_M and j - i < cap, where D is the
// linear regressor's fast metric bitlen(max d - min d) over the inner differences d_k = w_k -
// w_{k-1}. Starts go to a bitmap (the thread owns its chunk's words), then a popcount scan
// compacts them.
//
// Merge, round-synchronous: each round computes for every adjacent pair the size of the merged
// partition with the full regressor (S_M + len * b; pairs sorted by length onto a thread, a warp or a
// CTA each) and its gain over the two apart; every pair
// with a positive gain whose priority (gain, SplitMix64 of its start) beats both neighbouring
// pairs merges, all at once. Pair sizes are cached: only pairs touching a partition merged in the
// previous round are refitted. Rounds repeat until none merges.
#include <math.h>

#include <map>
#include <type_traits>
#include <vector>

#include "fit.cuh"
#include "leco_internal.cuh"
#include "var_partition.cuh"

namespace leco {

cudaError_t scan_u64(const uint64_t* in, uint64_t count, uint64_t* out, uint64_t* scratch,
                     uint64_t* total, cudaStream_t st);

namespace {

constexpr uint64_t kChunk = 1ull << 16;
constexpr uint64_t kNone = ~0ull;        // no merged size (pair longer than the cap)
constexpr uint32_t kLongPair = 1u << 14; // pairs longer than this are fitted by a whole CTA

// One chunk's greedy sweep. NARROW: every value of the chunk lies in (-2^62, 2^62) as int64, so the
// differences and their running extremes fit 64 bits (their range below 2^64, taken unsigned);
// otherwise 128-bit. The threshold test C <= tau S_M is done on integers: for an integer C and a
// real t, C <= t exactly when C <= floor(t). Values are read eight at a time ahead of the sweep's
// dependency chain.
template <bool NARROW, typename T>
__device__ __forceinline__ void split_chunk(const T* __restrict__ v, uint64_t a, uint64_t e, uint32_t cap,
                                            int64_t tfloor, uint64_t* __restrict__ bitmap) {
  using D = typename std::conditional<NARROW, int64_t, i128>::type;
  uint64_t i = a;
  uint64_t word = 1ull;  // position a opens a partition (a % 64 == 0)
  uint64_t wi = a >> 6;
  int64_t prev = (int64_t)v[a];
  D dmax = 0, dmin = 0;
  int cur = 0;
  int64_t nxt[8];  // the next batch, loaded while the current one is swept
#pragma unroll
  for (int u = 0; u < 8; u++) nxt[u] = a + 1 + u < e ? (int64_t)__ldg(v + a + 1 + u) : 0;
  for (uint64_t j0 = a + 1; j0 < e; j0 += 8) {
    int64_t buf[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      buf[u] = nxt[u];
      nxt[u] = j0 + 8 + u < e ? (int64_t)__ldg(v + j0 + 8 + u) : 0;
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const uint64_t j = j0 + u;
      if (j >= e) break;
      if ((j & 63) == 0) {
        bitmap[wi++] = word;
        word = 0;
      }
      const int64_t w = buf[u];
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
        if (NARROW)
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
        word |= 1ull << (j & 63);
        i = j;
        cur = 0;
        dmax = 0;
        dmin = 0;
      }
      prev = w;
    }
  }
  bitmap[wi] = word;
}

// Seeded split (§3.2.2, selecting good starting positions): the greedy sweep over the count values
// u_k = v[base + dir k] (dir = +1, or -1 to read them backwards); a partition opens at u-index k when
// u_k is refused, and mark(k) records it (the first partition, at k = 0, is not marked). Same rule,
// cap and integer threshold as split_chunk; values are read eight ahead of the dependency chain.
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

// narrow[c] = every value of chunk c lies in (-2^62, 2^62) as int64 (a CTA per chunk)
template <typename T>
__global__ void k_chunk_narrow(const T* __restrict__ v, uint64_t n, uint8_t* __restrict__ narrow) {
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  const int64_t lim = (int64_t)1 << 62;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t a = c * kChunk, e = min(a + kChunk, n);
    int bad = 0;
    if (sizeof(T) == 8)
      for (uint64_t j = a + threadIdx.x; j < e; j += blockDim.x) {
        const int64_t w = (int64_t)__ldg(v + j);
        bad |= (w <= -lim || w >= lim) ? 1 : 0;
      }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) narrow[c] = bad ? 0 : 1;
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

// seeds: nullptr for the left-to-right split, else each chunk's seed (k_chunk_seed)
template <typename T>
__global__ void k_split(const T* __restrict__ values, uint64_t n, uint32_t cap, int64_t tfloor,
                        const uint8_t* __restrict__ narrow, const uint64_t* __restrict__ seeds,
                        uint64_t* __restrict__ bitmap) {
  const uint64_t nchunks = (n + kChunk - 1) / kChunk;
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = c * kChunk;
    const uint64_t e = min(a + kChunk, n);
    if (seeds) {
      if (narrow[c])
        split_chunk_seeded<true>(values, a, e, seeds[c], cap, tfloor, bitmap);
      else
        split_chunk_seeded<false>(values, a, e, seeds[c], cap, tfloor, bitmap);
    } else if (narrow[c]) {
      split_chunk<true>(values, a, e, cap, tfloor, bitmap);
    } else {
      split_chunk<false>(values, a, e, cap, tfloor, bitmap);
    }
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

// Sizes S_M + len * b of spans [st[j], st[j + w]) (w = 1: partitions; w = 2: adjacent pairs) by the
// full fit. The spans to fit are first sorted into three work lists by length, so that each is fitted
// by a group of matching size: one thread for short spans (32 of them share a warp, and with it the
// single-lane parameter solve), a warp for medium ones, a CTA for long ones. A list's order is free:
// every span's size is independent of the others.
constexpr uint32_t kTinySpan = 256;

struct SpanLists {
  uint64_t* tiny;       // [0, counts[0])
  uint64_t* medium;     // [0, counts[1])
  uint64_t* lng;        // [0, counts[2])
  unsigned long long* counts;
};

// append j to list k with one atomic per warp and list
__device__ __forceinline__ void list_push(const SpanLists& L, int k, bool take, uint64_t j) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t mask = __ballot_sync(0xffffffffu, take);
  if (!mask) return;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if ((int)lane == leader) base = atomicAdd(&L.counts[k], (unsigned long long)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (take) {
    uint64_t* list = k == 0 ? L.tiny : (k == 1 ? L.medium : L.lng);
    list[base + __popc(mask & ((1u << lane) - 1u))] = j;
  }
}

// dirty == nullptr: every span. A span longer than cap gets no fit (out[j] = kNone).
__global__ void k_classify(const uint64_t* __restrict__ st, uint64_t count, uint32_t w, uint32_t cap,
                           const uint8_t* __restrict__ dirty, uint64_t* __restrict__ out, SpanLists L) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j0 = blockIdx.x * (uint64_t)blockDim.x; j0 < count; j0 += stride) {
    const uint64_t j = j0 + threadIdx.x;  // whole warps iterate together (list_push is warp-wide)
    bool t = false, md = false, lg = false;
    if (j < count && (!dirty || dirty[j])) {
      const uint64_t len = st[j + w] - st[j];
      if (len > cap)
        out[j] = kNone;
      else
        (len <= kTinySpan ? t : (len <= kLongPair ? md : lg)) = true;
    }
    list_push(L, 0, t, j);
    list_push(L, 1, md, j);
    list_push(L, 2, lg, j);
  }
}

__global__ void k_span_size_thread(const void* __restrict__ values, int dtype, const uint64_t* __restrict__ st,
                                   uint32_t w, int model, SpanLists L, uint64_t* __restrict__ out) {
  const uint64_t cnt = L.counts[0];
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = L.tiny[i];
    const uint64_t a = st[j], len = st[j + w] - a;
    const FitResult R = fit_range<1>(values, dtype, a, (uint32_t)len, model, 0, nullptr);
    out[j] = kSmBits + len * (uint64_t)R.b;
  }
}

__global__ void k_span_size_warp(const void* __restrict__ values, int dtype, const uint64_t* __restrict__ st,
                                 uint32_t w, int model, SpanLists L, uint64_t* __restrict__ out) {
  const uint64_t cnt = L.counts[1];
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = warp; i < cnt; i += nw) {
    const uint64_t j = L.medium[i];
    const uint64_t a = st[j], len = st[j + w] - a;
    const FitResult R = fit_range<32>(values, dtype, a, (uint32_t)len, model, threadIdx.x & 31u, nullptr);
    if ((threadIdx.x & 31u) == 0) out[j] = kSmBits + len * (uint64_t)R.b;
  }
}

__global__ void __launch_bounds__(256)
    k_span_size_block(const void* __restrict__ values, int dtype, const uint64_t* __restrict__ st, uint32_t w,
                      int model, SpanLists L, uint64_t* __restrict__ out) {
  __shared__ FitShared sm;
  const uint64_t cnt = L.counts[2];
  for (uint64_t i = blockIdx.x; i < cnt; i += gridDim.x) {
    const uint64_t j = L.lng[i];
    const uint64_t a = st[j], len = st[j + w] - a;
    const FitResult R = fit_range<256>(values, dtype, a, (uint32_t)len, model, threadIdx.x, &sm);
    if (threadIdx.x == 0) out[j] = kSmBits + len * (uint64_t)R.b;
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

__global__ void k_select(const uint64_t* __restrict__ st, const uint64_t* __restrict__ sz,
                         const uint64_t* __restrict__ msz, uint64_t m, uint8_t* __restrict__ sel,
                         unsigned long long* __restrict__ nsel) {
  uint32_t local = 0;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j + 1 < m;
       j += (uint64_t)gridDim.x * blockDim.x) {
    int64_t g;
    bool ok = pair_gain(sz, msz, j, &g) && g > 0;
    if (ok && j > 0) {
      int64_t gl;
      if (pair_gain(sz, msz, j - 1, &gl) && !beats(g, st[j], gl, st[j - 1])) ok = false;
    }
    if (ok && j + 2 < m) {
      int64_t gr;
      if (pair_gain(sz, msz, j + 1, &gr) && !beats(g, st[j], gr, st[j + 1])) ok = false;
    }
    sel[j] = ok ? 1 : 0;
    local += ok ? 1u : 0u;
  }
  local = (uint32_t)warp_sum_u64(local);
  if ((threadIdx.x & 31u) == 0 && local) atomicAdd(nsel, (unsigned long long)local);
}

// partition p survives unless it was merged into its left neighbour
__global__ void k_keep(const uint8_t* __restrict__ sel, uint64_t m, uint64_t* __restrict__ keep) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
       p += (uint64_t)gridDim.x * blockDim.x)
    keep[p] = (p == 0 || !sel[p - 1]) ? 1ull : 0ull;
}

__global__ void k_compact(const uint64_t* __restrict__ st, const uint64_t* __restrict__ sz,
                          const uint64_t* __restrict__ msz, const uint8_t* __restrict__ sel,
                          const uint64_t* __restrict__ newidx, uint64_t m, uint64_t n, uint64_t new_m,
                          uint64_t* __restrict__ nst, uint64_t* __restrict__ nsz,
                          uint64_t* __restrict__ nmsz, uint8_t* __restrict__ ndirty) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
       p += (uint64_t)gridDim.x * blockDim.x) {
    if (p > 0 && sel[p - 1]) continue;  // absorbed by p-1
    const uint64_t k = newidx[p];
    const bool mp = p + 1 < m && sel[p];
    nst[k] = st[p];
    nsz[k] = mp ? msz[p] : sz[p];
    const uint64_t q = mp ? p + 2 : p + 1;  // next surviving partition
    if (q < m) {
      const bool mq = q + 1 < m && sel[q];
      const bool d = mp || mq;
      ndirty[k] = d ? 1 : 0;
      if (!d) nmsz[k] = msz[p];
    }
    if (k == 0) nst[new_m] = n;
  }
}

__global__ void k_fill_u8(uint8_t* p, uint64_t count, uint8_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count;
       i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

int grid_for(uint64_t items, int per_block, int max_blocks_per_sm) {
  const uint64_t need = (items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)sm_count() * max_blocks_per_sm;
  return (int)(need < cap ? (need ? need : 1) : cap);
}

template <typename T>
cudaError_t dalloc(T** p, uint64_t elems, cudaStream_t st) {
  return dev_alloc((void**)p, (elems ? elems : 1) * sizeof(T), st);
}

// spans longer than kLongPair among those of a column of n values: partitions are disjoint, and
// of adjacent pairs every other one is
inline uint64_t long_span_cap(uint64_t n) { return 2 * (n / kLongPair + 1); }

// sizes of the `count` spans [st[j], st[j + w]) selected by dirty (nullptr: all) into out; the lists
// hold `count` entries each (tiny, medium) and long_span_cap(n) (long)
cudaError_t span_sizes(const void* values, int dtype, uint64_t n, const uint64_t* st, uint64_t count, uint32_t w,
                       uint32_t cap, int model, const uint8_t* dirty, uint64_t* out, const SpanLists& L,
                       cudaStream_t stm) {
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(L.counts, 0, 3 * sizeof(unsigned long long), stm);
  if (e != cudaSuccess) return e;
  k_classify<<<grid_for(count, 256, 8), 256, 0, stm>>>(st, count, w, cap, dirty, out, L);
  k_span_size_thread<<<grid_for(count, 256, 8), 256, 0, stm>>>(values, dtype, st, w, model, L, out);
  k_span_size_warp<<<grid_for(count * 32, 256, 8), 256, 0, stm>>>(values, dtype, st, w, model, L, out);
  k_span_size_block<<<grid_for(long_span_cap(n), 1, 4), 256, 0, stm>>>(values, dtype, st, w, model, L, out);
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

// Runs split + merge; writes m+1 starts to starts_out (capacity n+1) and m to *m_out.
cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap,
                          int model, bool seeded, uint64_t* starts_out, uint64_t* m_out, cudaStream_t st) {
  *m_out = 0;
  if (n == 0) {
    const uint64_t zero = 0;
    cudaError_t e = cudaMemcpyAsync(starts_out, &zero, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
  }
  const double thresh = tau * (double)kSmBits;
  const uint64_t nw = (n + 63) / 64;
  uint64_t *bitmap = nullptr, *cnt = nullptr, *pos = nullptr, *scan_scratch = nullptr, *d_total = nullptr;
  uint64_t* seeds = nullptr;
  cudaError_t e = cudaSuccess;
  const uint64_t scan_elems = nw / 2048 + 2;
#define LECO_TRY(x)          \
  do {                       \
    e = (x);                 \
    if (e != cudaSuccess) goto done; \
  } while (0)
  {
    LECO_TRY(dalloc(&bitmap, nw, st));
    LECO_TRY(dalloc(&cnt, nw, st));
    LECO_TRY(dalloc(&pos, nw, st));
    LECO_TRY(dalloc(&scan_scratch, scan_elems + 1, st));
    LECO_TRY(dalloc(&d_total, 1, st));
    const uint64_t nchunks = (n + kChunk - 1) / kChunk;
    // C <= tau * S_M for an integer C: C <= floor(tau * S_M) (thresh >= 0, below 2^62 here). The
    // sweeps are serial per chunk, so each gets a warp of its own SM slot (one-warp blocks)
    const int64_t tfloor = thresh < 4.0e18 ? (int64_t)floor(thresh) : INT64_MAX;
    uint8_t* narrow = reinterpret_cast<uint8_t*>(cnt);  // scratch: cnt is not used until the popcount
    if (seeded) LECO_TRY(dalloc(&seeds, nchunks, st));
    if (dtype == LECO_U32) {
      k_chunk_narrow<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(static_cast<const uint32_t*>(values), n, narrow);
      if (seeded)
        k_chunk_seed<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(static_cast<const uint32_t*>(values), n, seeds);
      k_split<<<grid_for(nchunks, 32, 32), 32, 0, st>>>(static_cast<const uint32_t*>(values), n, cap, tfloor, narrow,
                                                         seeds, bitmap);
    } else {
      k_chunk_narrow<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(static_cast<const uint64_t*>(values), n, narrow);
      if (seeded)
        k_chunk_seed<<<grid_for(nchunks, 1, 8), 256, 0, st>>>(static_cast<const uint64_t*>(values), n, seeds);
      k_split<<<grid_for(nchunks, 32, 32), 32, 0, st>>>(static_cast<const uint64_t*>(values), n, cap, tfloor, narrow,
                                                         seeds, bitmap);
    }
    LECO_TRY(cudaGetLastError());
    k_popc<<<grid_for(nw, 256, 8), 256, 0, st>>>(bitmap, nw, cnt);
    LECO_TRY(cudaGetLastError());
    LECO_TRY(scan_u64(cnt, nw, pos, scan_scratch, d_total, st));
    uint64_t m = 0;
    LECO_TRY(cudaMemcpyAsync(&m, d_total, 8, cudaMemcpyDeviceToHost, st));
    LECO_TRY(cudaStreamSynchronize(st));
    k_scatter_starts<<<grid_for(nw, 256, 8), 256, 0, st>>>(bitmap, nw, pos, n, m, starts_out);
    LECO_TRY(cudaGetLastError());
    cudaFreeAsync(cnt, st);
    cnt = nullptr;
    cudaFreeAsync(pos, st);
    pos = nullptr;
    cudaFreeAsync(bitmap, st);
    bitmap = nullptr;
    if (seeds) cudaFreeAsync(seeds, st);
    seeds = nullptr;
    cudaFreeAsync(scan_scratch, st);
    scan_scratch = nullptr;

    // merge state (ping-pong)
    uint64_t *st_b = nullptr, *sz_a = nullptr, *sz_b = nullptr, *msz_a = nullptr, *msz_b = nullptr;
    uint64_t *keep = nullptr, *newidx = nullptr, *scr = nullptr;
    uint8_t *dirty_a = nullptr, *dirty_b = nullptr, *sel = nullptr;
    unsigned long long* d_nsel = nullptr;
    const uint64_t m0 = m;
    const uint64_t scr_elems = m0 / 2048 + 2;
    bool ok = true;
    ok = ok && dalloc(&st_b, m0 + 1, st) == cudaSuccess;
    ok = ok && dalloc(&sz_a, m0, st) == cudaSuccess && dalloc(&sz_b, m0, st) == cudaSuccess;
    ok = ok && dalloc(&msz_a, m0, st) == cudaSuccess && dalloc(&msz_b, m0, st) == cudaSuccess;
    ok = ok && dalloc(&keep, m0, st) == cudaSuccess && dalloc(&newidx, m0, st) == cudaSuccess;
    ok = ok && dalloc(&scr, scr_elems + 1, st) == cudaSuccess;
    ok = ok && dalloc(&dirty_a, m0, st) == cudaSuccess && dalloc(&dirty_b, m0, st) == cudaSuccess;
    ok = ok && dalloc(&sel, m0, st) == cudaSuccess && dalloc(&d_nsel, 1, st) == cudaSuccess;
    SpanLists lists;
    lists.tiny = lists.medium = lists.lng = nullptr;
    lists.counts = nullptr;
    ok = ok && dalloc(&lists.tiny, m0, st) == cudaSuccess && dalloc(&lists.medium, m0, st) == cudaSuccess;
    ok = ok && dalloc(&lists.lng, long_span_cap(n), st) == cudaSuccess && dalloc(&lists.counts, 3, st) == cudaSuccess;
    uint64_t* cur_st = starts_out;
    uint64_t* nxt_st = st_b;
    if (ok && m > 1) {
      e = span_sizes(values, dtype, n, cur_st, m, 1, ~0u, model, nullptr, sz_a, lists, st);
      k_fill_u8<<<grid_for(m, 256, 8), 256, 0, st>>>(dirty_a, m, 1);
      if (e == cudaSuccess) e = cudaGetLastError();
      while (e == cudaSuccess && m > 1) {
        e = span_sizes(values, dtype, n, cur_st, m - 1, 2, cap, model, dirty_a, msz_a, lists, st);
        if (e != cudaSuccess) break;
        cudaMemsetAsync(d_nsel, 0, 8, st);
        k_select<<<grid_for(m, 256, 8), 256, 0, st>>>(cur_st, sz_a, msz_a, m, sel, d_nsel);
        unsigned long long nsel = 0;
        e = cudaMemcpyAsync(&nsel, d_nsel, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || nsel == 0) break;
        k_keep<<<grid_for(m, 256, 8), 256, 0, st>>>(sel, m, keep);
        e = scan_u64(keep, m, newidx, scr, d_total, st);
        if (e != cudaSuccess) break;
        const uint64_t new_m = m - nsel;
        k_compact<<<grid_for(m, 256, 8), 256, 0, st>>>(cur_st, sz_a, msz_a, sel, newidx, m, n, new_m,
                                                       nxt_st, sz_b, msz_b, dirty_b);
        e = cudaGetLastError();
        uint64_t* t64;
        uint8_t* t8;
        t64 = cur_st; cur_st = nxt_st; nxt_st = t64;
        t64 = sz_a; sz_a = sz_b; sz_b = t64;
        t64 = msz_a; msz_a = msz_b; msz_b = t64;
        t8 = dirty_a; dirty_a = dirty_b; dirty_b = t8;
        m = new_m;
      }
      if (e == cudaSuccess && cur_st != starts_out)
        e = cudaMemcpyAsync(starts_out, cur_st, (m + 1) * 8, cudaMemcpyDeviceToDevice, st);
    } else if (!ok) {
      e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // st_b may be cur_st's partner; both are scratch except starts_out
    cudaFreeAsync(cur_st == starts_out ? nxt_st : cur_st, st);
    cudaFreeAsync(sz_a, st);
    cudaFreeAsync(sz_b, st);
    cudaFreeAsync(msz_a, st);
    cudaFreeAsync(msz_b, st);
    cudaFreeAsync(keep, st);
    cudaFreeAsync(newidx, st);
    cudaFreeAsync(scr, st);
    cudaFreeAsync(dirty_a, st);
    cudaFreeAsync(dirty_b, st);
    cudaFreeAsync(sel, st);
    cudaFreeAsync(d_nsel, st);
    cudaFreeAsync(lists.tiny, st);
    cudaFreeAsync(lists.medium, st);
    cudaFreeAsync(lists.lng, st);
    cudaFreeAsync(lists.counts, st);
    if (e == cudaSuccess) *m_out = m;
  }
done:
  if (seeds) cudaFreeAsync(seeds, st);
  if (bitmap) cudaFreeAsync(bitmap, st);
  if (cnt) cudaFreeAsync(cnt, st);
  if (pos) cudaFreeAsync(pos, st);
  if (scan_scratch) cudaFreeAsync(scan_scratch, st);
  if (d_total) cudaFreeAsync(d_total, st);
#undef LECO_TRY
  return e;
}

cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap,
                          int model, uint64_t* starts_out, uint64_t* m_out, cudaStream_t st) {
  return var_partition(values, dtype, n, tau, cap, model, false, starts_out, m_out, st);
}

}  // namespace leco
