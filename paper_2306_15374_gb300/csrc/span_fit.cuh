// Span fits of the variable partitioner (§3.1 Regressor over the spans of §3.2.2): the moments of a
// span's values and the cooperative passes that let several lanes work on one span.
//
// Moments of a span (w = the value as two's complement int64, x = the local index): T0 = sum w,
// T1 = sum x w, and min and max of w. The fit's least-squares moment is S = sum (2x - (N-1)) w =
// 2 T1 - (N-1) T0, and two adjacent spans' moments combine exactly (the right span's x shifts by
// the left span's length: T1 gains N_left T0_right).
#pragma once

#include "fit.cuh"
#include "leco_internal.cuh"

namespace leco {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

struct SpanStats {
  i128 T0;
  i128 T1;
  int64_t mn;
  int64_t mx;
};

__device__ __forceinline__ SpanStats combine_stats(const SpanStats& l, uint64_t nl, const SpanStats& r) {
  SpanStats c;
  c.T0 = l.T0 + r.T0;
  c.T1 = l.T1 + r.T1 + mul_i128_u64(r.T0, nl);
  c.mn = min(l.mn, r.mn);
  c.mx = max(l.mx, r.mx);
  return c;
}

// reductions over aligned tiles of TILE lanes (32: the warp) whose result every lane of the tile
// receives
template <int TILE = 32>
__device__ __forceinline__ int64_t xw_min(int64_t v) {
  for (int o = TILE / 2; o > 0; o >>= 1) v = min(v, (int64_t)__shfl_xor_sync(kFull, v, o));
  return v;
}
template <int TILE = 32>
__device__ __forceinline__ int64_t xw_max(int64_t v) {
  for (int o = TILE / 2; o > 0; o >>= 1) v = max(v, (int64_t)__shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ uint64_t xw_min_u(uint64_t v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, (uint64_t)__shfl_xor_sync(kFull, v, o));
  return v;
}
template <int TILE = 32>
__device__ __forceinline__ uint64_t xw_max_u(uint64_t v) {
  for (int o = TILE / 2; o > 0; o >>= 1) v = max(v, (uint64_t)__shfl_xor_sync(kFull, v, o));
  return v;
}
template <int TILE = 32>
__device__ __forceinline__ i128 xw_sum(i128 v) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
  for (int o = TILE / 2; o > 0; o >>= 1) {
    const uint64_t l2 = __shfl_xor_sync(kFull, lo, o);
    const uint64_t h2 = __shfl_xor_sync(kFull, hi, o);
    const uint64_t nl = lo + l2;
    hi = hi + h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  return (i128)(((u128)hi << 64) | lo);
}

// moments of the positions x, x + step, ... < N of the span whose first value is p[0]
template <typename T>
__device__ __forceinline__ SpanStats stats_part(const T* p, uint32_t x, uint32_t N, uint32_t step) {
  SpanStats s;
  s.T0 = 0;
  s.T1 = 0;
  s.mn = INT64_MAX;
  s.mx = INT64_MIN;
#pragma unroll 8
  for (; x < N; x += step) {
    const int64_t w = (int64_t)p[x];
    s.mn = min(s.mn, w);
    s.mx = max(s.mx, w);
    s.T0 += (i128)w;
    s.T1 += mul_s64(w, (int64_t)x);
  }
  return s;
}

// residual range at the positions x, x + step, ... < N under the parameters P (fit.cuh, steps 4
// and the fallback's widest zigzag residual), accumulated into lo, hi, zmax
template <typename T>
__device__ __forceinline__ void resid_part(const T* p, uint32_t x, uint32_t N, uint32_t step, const FitParams& P,
                                           int64_t& lo, int64_t& hi, uint64_t& zmax) {
  if (P.fallback) {
#pragma unroll 4
    for (; x < N; x += step) zmax = max(zmax, zz_encode((int64_t)((uint64_t)p[x] - (uint64_t)P.fb_shift)));
    return;
  }
  uint64_t F = (uint64_t)P.B * x;
  const uint64_t dF = (uint64_t)P.B * step;
  if (P.s >= 0) {
#pragma unroll 8
    for (; x < N; x += step, F += dF) {
      const int64_t r = (int64_t)p[x] - ((int64_t)F >> P.s);
      lo = min(lo, r);
      hi = max(hi, r);
    }
  } else {
#pragma unroll 4
    for (; x < N; x += step, F += dF) {
      const int64_t r = (int64_t)p[x] - (int64_t)(F << (-P.s));
      lo = min(lo, r);
      hi = max(hi, r);
    }
  }
}

__device__ __forceinline__ FitParams shfl_params(const FitParams& P, int src) {
  FitParams q;
  q.B = (int64_t)__shfl_sync(kFull, (unsigned long long)P.B, src);
  q.fb_shift = (int64_t)__shfl_sync(kFull, (unsigned long long)P.fb_shift, src);
  q.s = __shfl_sync(kFull, P.s, src);
  q.fallback = __shfl_sync(kFull, P.fallback, src);
  return q;
}

// Spans fitted cooperatively: the spans of the lanes set in mask, TILE lanes each (32 / TILE spans
// at a time, in the order of their lanes). Each call hands every owning lane the reduced result of
// its own span. p, N, P: the calling lane's span (a pointer to its first value, in global or shared
// memory, its length and its parameters).
template <int TILE, typename T>
__device__ __forceinline__ void coop_stats(uint32_t mask, const T* p, uint32_t N, SpanStats& S) {
  constexpr int NT = 32 / TILE;
  const int lane = (int)(threadIdx.x & 31u), tile = lane / TILE, r = lane % TILE;
  const int total = __popc(mask);
  const bool mine = (mask >> lane) & 1u;
  const int rank = __popc(mask & ((1u << lane) - 1u));
  for (int it = 0; it * NT < total; it++) {
    const int k = it * NT + tile;
    const int sl = k < total ? (int)__fns(mask, 0, k + 1) : lane;
    const T* ps = reinterpret_cast<const T*>(__shfl_sync(kFull, (unsigned long long)p, sl));
    const uint32_t Ns = __shfl_sync(kFull, N, sl);
    SpanStats q = stats_part(ps, (uint32_t)r, k < total ? Ns : 0u, (uint32_t)TILE);
    q.T0 = xw_sum<TILE>(q.T0);
    q.T1 = xw_sum<TILE>(q.T1);
    q.mn = xw_min<TILE>(q.mn);
    q.mx = xw_max<TILE>(q.mx);
    const bool take = mine && rank / NT == it;
    const int src = take ? (rank % NT) * TILE : lane;
    const uint64_t t0l = __shfl_sync(kFull, (uint64_t)q.T0, src), t0h = __shfl_sync(kFull, (uint64_t)((u128)q.T0 >> 64), src);
    const uint64_t t1l = __shfl_sync(kFull, (uint64_t)q.T1, src), t1h = __shfl_sync(kFull, (uint64_t)((u128)q.T1 >> 64), src);
    const int64_t mn = __shfl_sync(kFull, q.mn, src), mx = __shfl_sync(kFull, q.mx, src);
    if (take) {
      S.T0 = (i128)(((u128)t0h << 64) | t0l);
      S.T1 = (i128)(((u128)t1h << 64) | t1l);
      S.mn = mn;
      S.mx = mx;
    }
  }
}

template <int TILE, typename T>
__device__ __forceinline__ void coop_resid(uint32_t mask, const T* p, uint32_t N, const FitParams& P, int64_t& lo,
                                           int64_t& hi, uint64_t& zmax) {
  constexpr int NT = 32 / TILE;
  const int lane = (int)(threadIdx.x & 31u), tile = lane / TILE, r = lane % TILE;
  const int total = __popc(mask);
  const bool mine = (mask >> lane) & 1u;
  const int rank = __popc(mask & ((1u << lane) - 1u));
  for (int it = 0; it * NT < total; it++) {
    const int k = it * NT + tile;
    const int sl = k < total ? (int)__fns(mask, 0, k + 1) : lane;
    const T* ps = reinterpret_cast<const T*>(__shfl_sync(kFull, (unsigned long long)p, sl));
    const uint32_t Ns = __shfl_sync(kFull, N, sl);
    const FitParams Ps = shfl_params(P, sl);
    int64_t l = INT64_MAX, h = INT64_MIN;
    uint64_t z = 0;
    resid_part(ps, (uint32_t)r, k < total ? Ns : 0u, (uint32_t)TILE, Ps, l, h, z);
    l = xw_min<TILE>(l);
    h = xw_max<TILE>(h);
    z = xw_max_u<TILE>(z);
    const bool take = mine && rank / NT == it;
    const int src = take ? (rank % NT) * TILE : lane;
    l = __shfl_sync(kFull, l, src);
    h = __shfl_sync(kFull, h, src);
    z = __shfl_sync(kFull, z, src);
    if (take) {
      lo = l;
      hi = h;
      zmax = z;
    }
  }
}


constexpr uint32_t kLaneSpan = 64;     // a lane fits spans up to this long on its own
constexpr uint32_t kTileSpan = 1024;   // eight lanes fit longer spans up to this long, four at a time

}  // namespace
}  // namespace leco
