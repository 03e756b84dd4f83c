// Partition fit shared by the encoder and the variable-length partitioner (§3.1 Regressor).
//
// Fit of one partition of N values (w = the value as two's complement int64):
//  1. exact least-squares slope q = 6S/D, S = sum (2x - (N-1)) (w_x - w_0), D = N (N^2 - 1)
//     (integer moments reduced across the group in int128; q = 0 for the constant model);
//  2. magnitude bound U = max|w| + (wmax - wmin) + (ceil|q| + 1) N + 4; bitlen(U) > 62 falls back
//     to the constant model on the grid 2^11 (residuals taken mod 2^64);
//  3. grid exponent s = min(52, 52 - bitlen(U)), slope B = round(q 2^s) (half up);
//  4. residual range [lo, hi] of r0_x = w_x - floor(B x 2^-s) (a second pass);
//  5. minimax intercept t = lo + ceil((hi - lo)/2), rounded down to the grid step 2^max(0,-s);
//  6. width b = bitlen(max(zigzag(lo - t), zigzag(hi - t))) (zigzag is V-shaped, so the extremes
//     of the residual range carry the maximum).
// The bound makes theta0 = A 2^-s and theta1 = B 2^-s exact binary64 numbers whose prediction
// floor(fl(fl(theta1 x) + theta0)) equals the integer (A + B x) >> s for every x < N.
#pragma once

#include "leco_internal.cuh"

namespace leco {
namespace {



__device__ __forceinline__ i128 floordiv_i128(i128 num, i128 den) {  // den > 0
  i128 q = num / den;
  if ((num % den) != 0 && num < 0) q -= 1;
  return q;
}

__device__ __forceinline__ i128 round_half_up_i128(i128 num, i128 den) {  // den > 0
  return floordiv_i128(2 * num + den, 2 * den);
}

__device__ __forceinline__ double pow2(int e) {  // exact 2^e for -1022 <= e <= 1023
  return __longlong_as_double((long long)(1023 + e) << 52);
}

struct FitParams {
  int64_t B;
  int64_t fb_shift;  // fallback: theta0 as an integer (multiple of 2^11)
  int32_t s;
  int32_t fallback;
};

struct FitResult {
  double theta0;
  double theta1;
  int32_t s;
  uint32_t b;
};

// step 1-3 (one thread): parameters from the reduced moments
__device__ FitParams solve_params(i128 S, int64_t mx, int64_t mn, uint32_t N, bool lin) {
  FitParams P;
  const i128 D = lin ? (i128)N * ((i128)N * (i128)N - 1) : (i128)1;
  const i128 sixS = lin ? 6 * S : (i128)0;
  const i128 a6 = sixS < 0 ? -sixS : sixS;
  const i128 Q = (a6 + D - 1) / D;
  const i128 amx = mx < 0 ? -(i128)mx : (i128)mx;
  const i128 amn = mn < 0 ? -(i128)mn : (i128)mn;
  const i128 M = amx > amn ? amx : amn;
  const i128 U = M + ((i128)mx - (i128)mn) + (Q + 1) * (i128)N + 4;
  const int eU = bitlen_u128((u128)U);
  if (eU > 62) {
    const i128 t = (i128)mn + (((i128)mx - (i128)mn + 1) / 2);
    const i128 tg = floordiv_i128(t, (i128)2048);
    P.fallback = 1;
    P.s = -11;
    P.B = 0;
    P.fb_shift = (int64_t)(tg * 2048);
    return P;
  }
  int s = 52 - eU;
  if (s > 52) s = 52;
  i128 B = 0;
  if (lin) {
    if (s >= 0)
      B = round_half_up_i128(sixS * ((i128)1 << s), D);
    else
      B = round_half_up_i128(sixS, D * ((i128)1 << (-s)));
  }
  P.fallback = 0;
  P.s = s;
  P.B = (int64_t)B;
  P.fb_shift = 0;
  return P;
}

// steps 5-6 (one thread)
__device__ FitResult finish_fit(const FitParams& P, int64_t lo, int64_t hi, uint64_t fb_maxzz) {
  FitResult R;
  if (P.fallback) {
    R.theta0 = (double)P.fb_shift;  // multiple of 2^11 with |.| <= 2^63: exact
    R.theta1 = 0.0;
    R.s = -11;
    R.b = (uint32_t)bitlen_u64(fb_maxzz);
    return R;
  }
  const int s = P.s;
  const i128 t = (i128)lo + (((i128)hi - (i128)lo + 1) / 2);
  i128 shift, A;
  if (s >= 0) {
    shift = t;
    A = t * ((i128)1 << s);
  } else {
    const i128 tg = floordiv_i128(t, (i128)1 << (-s));
    shift = tg * ((i128)1 << (-s));
    A = tg;
  }
  const int64_t lo2 = (int64_t)((i128)lo - shift), hi2 = (int64_t)((i128)hi - shift);
  const uint64_t z = max(zz_encode(lo2), zz_encode(hi2));
  R.b = (uint32_t)bitlen_u64(z);
  R.s = s;
  R.theta0 = (double)(int64_t)A * pow2(-s);
  R.theta1 = (double)P.B * pow2(-s);
  return R;
}

__device__ __forceinline__ int64_t line_at(int64_t B, int32_t s, uint32_t x) {
  const int64_t bx = B * (int64_t)x;
  return s >= 0 ? (bx >> s) : (bx << (-s));
}

// Group fit: GROUP threads (a warp, or a whole CTA when GROUP > 32) fit [a, a+N). Returns the
// result in every thread of the group. sm: shared scratch (only used when GROUP > 32).
struct FitShared {
  i128 S[32];
  int64_t mx[32], mn[32];
  uint64_t zmax[32];
  FitParams P;
  FitResult R;
};

template <int GROUP>
__device__ FitResult fit_range(const void* __restrict__ values, int dtype, uint64_t a, uint32_t N,
                               int model, uint32_t rank, FitShared* sm) {
  const bool lin = model == LECO_MODEL_LINEAR && N >= 2;
  const int64_t w0 = (int64_t)load_value(values, dtype, a);
  i128 S = 0;
  int64_t mx = INT64_MIN, mn = INT64_MAX;
  const int64_t nm1 = (int64_t)N - 1;
  for (uint32_t x = rank; x < N; x += GROUP) {
    const int64_t w = (int64_t)load_value(values, dtype, a + x);
    mx = max(mx, w);
    mn = min(mn, w);
    if (lin) {
      const int64_t u = 2 * (int64_t)x - nm1;
      S += (i128)u * ((i128)w - (i128)w0);
    }
  }
  S = warp_sum_i128(S);
  mx = warp_max_i64(mx);
  mn = warp_min_i64(mn);
  const uint32_t lane = rank & 31u;
  FitParams P;
  if (GROUP == 32) {
    if (lane == 0) P = solve_params(S, mx, mn, N, lin);
    P.B = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)P.B, 0);
    P.fb_shift = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)P.fb_shift, 0);
    P.s = __shfl_sync(0xffffffffu, P.s, 0);
    P.fallback = __shfl_sync(0xffffffffu, P.fallback, 0);
  } else {
    const uint32_t wid = rank >> 5;
    if (lane == 0) {
      sm->S[wid] = S;
      sm->mx[wid] = mx;
      sm->mn[wid] = mn;
    }
    __syncthreads();
    if (rank == 0) {
      for (int k = 1; k < GROUP / 32; k++) {
        S += sm->S[k];
        mx = max(mx, sm->mx[k]);
        mn = min(mn, sm->mn[k]);
      }
      sm->P = solve_params(S, mx, mn, N, lin);
    }
    __syncthreads();
    P = sm->P;
  }

  // pass 2
  int64_t lo = INT64_MAX, hi = INT64_MIN;
  uint64_t zmax = 0;
  if (P.fallback) {
    for (uint32_t x = rank; x < N; x += GROUP) {
      const uint64_t v = load_value(values, dtype, a + x);
      zmax = max(zmax, zz_encode((int64_t)(v - (uint64_t)P.fb_shift)));
    }
    zmax = warp_max_u64(zmax);
  } else {
    for (uint32_t x = rank; x < N; x += GROUP) {
      const int64_t w = (int64_t)load_value(values, dtype, a + x);
      const int64_t r = w - line_at(P.B, P.s, x);
      lo = min(lo, r);
      hi = max(hi, r);
    }
    lo = warp_min_i64(lo);
    hi = warp_max_i64(hi);
  }
  FitResult R;
  if (GROUP == 32) {
    if (lane == 0) R = finish_fit(P, lo, hi, zmax);
    R.theta0 = __shfl_sync(0xffffffffu, R.theta0, 0);
    R.theta1 = __shfl_sync(0xffffffffu, R.theta1, 0);
    R.s = __shfl_sync(0xffffffffu, R.s, 0);
    R.b = __shfl_sync(0xffffffffu, R.b, 0);
  } else {
    const uint32_t wid = rank >> 5;
    if (lane == 0) {
      sm->mx[wid] = hi;
      sm->mn[wid] = lo;
      sm->zmax[wid] = zmax;
    }
    __syncthreads();
    if (rank == 0) {
      for (int k = 1; k < GROUP / 32; k++) {
        hi = max(hi, sm->mx[k]);
        lo = min(lo, sm->mn[k]);
        zmax = max(zmax, sm->zmax[k]);
      }
      sm->R = finish_fit(P, lo, hi, zmax);
    }
    __syncthreads();
    R = sm->R;
    __syncthreads();  // sm is reused by the next partition
  }
  return R;
}

}  // namespace
}  // namespace leco
