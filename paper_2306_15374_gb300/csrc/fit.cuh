// Partition fit shared by the encoder and the variable-length partitioner (§3.1 Regressor).
//
// Fit of one partition of N values (w = the value as two's complement int64):
//  1. exact least-squares slope q = 6S/D, S = sum (2x - (N-1)) (w_x - w_0), D = N (N^2 - 1)
//     (integer moments reduced across the group in int128; q = 0 for the constant model; the
//     divisions are exact 128-by-64 long divisions where the divisor allows, see floordiv_i128);
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



// (u1 2^64 + u0) / v for u1 < v (so the quotient fits 64 bits), with the remainder: schoolbook
// long division in base 2^32 after normalising v (Knuth's algorithm D with two quotient digits, in
// the form of Warren's "divlu", Hacker's Delight §9-4). Each digit is estimated from the top two
// dividend digits over the top divisor digit and corrected at most twice.
__host__ __device__ __forceinline__ uint64_t divlu(uint64_t u1, uint64_t u0, uint64_t v, uint64_t* rem) {
  const uint64_t base = 1ull << 32;
#ifdef __CUDA_ARCH__
  const int sh = __clzll((long long)v);  // v > 0
#else
  const int sh = __builtin_clzll(v);
#endif
  v <<= sh;
  const uint64_t vn1 = v >> 32, vn0 = v & 0xFFFFFFFFull;
  const uint64_t un32 = sh ? (u1 << sh) | (u0 >> (64 - sh)) : u1;
  const uint64_t un10 = u0 << sh;
  const uint64_t un1 = un10 >> 32, un0 = un10 & 0xFFFFFFFFull;
  uint64_t q1 = un32 / vn1, rhat = un32 - q1 * vn1;
  while (q1 >= base || q1 * vn0 > base * rhat + un1) {
    q1--;
    rhat += vn1;
    if (rhat >= base) break;
  }
  const uint64_t un21 = un32 * base + un1 - q1 * v;
  uint64_t q0 = un21 / vn1;
  rhat = un21 - q0 * vn1;
  while (q0 >= base || q0 * vn0 > base * rhat + un0) {
    q0--;
    rhat += vn1;
    if (rhat >= base) break;
  }
  *rem = (un21 * base + un0 - q0 * v) >> sh;
  return q1 * base + q0;
}

// floor(num / den) for den > 0, exactly. Divisors below 2^64 (every fit of a partition up to 2^21
// values) take two native 64-bit divisions and one 128-by-64 long division; wider divisors use
// the generic 128-bit routine, whose bit-serial latency would otherwise stall a whole CTA per
// fitted partition.
__host__ __device__ __forceinline__ i128 floordiv_i128(i128 num, i128 den) {
  if ((den >> 64) == 0 && num != ((i128)1 << 127)) {
    const uint64_t d = (uint64_t)den;
    const bool neg = num < 0;
    const u128 u = neg ? (u128)0 - (u128)num : (u128)num;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    const uint64_t qh = hi / d;
    uint64_t r = 0;
    const uint64_t ql = divlu(hi - qh * d, lo, d, &r);
    const u128 q = ((u128)qh << 64) | ql;
    return neg ? -(i128)q - (r != 0 ? 1 : 0) : (i128)q;
  }
  i128 t = num / den;
  if ((num % den) != 0 && num < 0) t -= 1;
  return t;
}

__host__ __device__ __forceinline__ i128 round_half_up_i128(i128 num, i128 den) {  // den > 0
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
  const i128 Q = floordiv_i128(a6 + D - 1, D);  // ceil(|6S| / D)
  const i128 amx = mx < 0 ? -(i128)mx : (i128)mx;
  const i128 amn = mn < 0 ? -(i128)mn : (i128)mn;
  const i128 M = amx > amn ? amx : amn;
  const i128 U = M + ((i128)mx - (i128)mn) + (Q + 1) * (i128)N + 4;
  const int eU = bitlen_u128((u128)U);
  if (eU > 62) {
    const i128 t = (i128)mn + (((i128)mx - (i128)mn + 1) / 2);
    const i128 tg = t >> 11;  // floor(t / 2^11)
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
    const i128 tg = t >> (-s);  // floor(t / 2^-s)
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


// Group fit: GROUP threads (one thread, a warp, or a whole CTA when GROUP > 32) fit [a, a+N).
// Returns the result in every thread of the group. sm: shared scratch (only used when GROUP > 32).
struct FitShared {
  i128 S[32];
  int64_t mx[32], mn[32];
  uint64_t zmax[32];
  FitParams P;
  FitResult R;
};

// Pass 1 over one group member's positions x = rank, rank + GROUP, ... < N of the values v (the
// partition's first value at v[0]): min, max and (linear model) S = sum u_x w_x with
// u_x = 2x - (N-1), where w is the value as two's complement int64. S equals
// sum u_x (w_x - w_0) because the u_x sum to zero. Each term is split as u w_hi 2^32 + u w_lo with
// 32 x 32 -> 64-bit products, accumulated in 64 bits over at most 64 terms (|u| < 2^24: each
// partial stays below 2^62), then folded into 128 bits.
template <int GROUP, typename T>
__device__ __forceinline__ void fit_pass1(const T* __restrict__ v, uint32_t N, bool lin, uint32_t rank, i128* S_out,
                                          int64_t* mx_out, int64_t* mn_out) {
  int64_t mx = INT64_MIN, mn = INT64_MAX;
  i128 S = 0;
  if (lin) {
    const int64_t nm1 = (int64_t)N - 1;
    for (uint32_t x0 = rank; x0 < N; x0 += 64u * GROUP) {
      const uint32_t xe = N - x0 > 64u * GROUP ? x0 + 64u * GROUP : N;
      int64_t acc_hi = 0, acc_lo = 0;
      int32_t u = (int32_t)(2 * (int64_t)x0 - nm1);
#pragma unroll 4
      for (uint32_t x = x0; x < xe; x += GROUP, u += 2 * GROUP) {
        const int64_t w = (int64_t)__ldg(v + x);
        mx = max(mx, w);
        mn = min(mn, w);
        if (sizeof(T) == 8) acc_hi += (int64_t)u * (int64_t)(int32_t)(w >> 32);
        acc_lo += (int64_t)u * (int64_t)(uint32_t)w;
      }
      S += (i128)acc_hi * ((i128)1 << 32) + (i128)acc_lo;
    }
  } else {
#pragma unroll 4
    for (uint32_t x = rank; x < N; x += GROUP) {
      const int64_t w = (int64_t)__ldg(v + x);
      mx = max(mx, w);
      mn = min(mn, w);
    }
  }
  *S_out = S;
  *mx_out = mx;
  *mn_out = mn;
}

// Pass 2: range [lo, hi] of the residuals w_x - line(x) with line(x) = (B x) >> s (s >= 0) or
// (B x) << -s, B x taken mod 2^64 and stepped by B GROUP from one position to the next.
template <int GROUP, typename T>
__device__ __forceinline__ void fit_pass2(const T* __restrict__ v, uint32_t N, int64_t B, int32_t s, uint32_t rank,
                                          int64_t* lo_out, int64_t* hi_out) {
  int64_t lo = INT64_MAX, hi = INT64_MIN;
  uint64_t F = (uint64_t)B * rank;
  const uint64_t dF = (uint64_t)B * GROUP;
  if (s >= 0) {
#pragma unroll 4
    for (uint32_t x = rank; x < N; x += GROUP, F += dF) {
      const int64_t r = (int64_t)__ldg(v + x) - ((int64_t)F >> s);
      lo = min(lo, r);
      hi = max(hi, r);
    }
  } else {
    for (uint32_t x = rank; x < N; x += GROUP, F += dF) {
      const int64_t r = (int64_t)__ldg(v + x) - (int64_t)(F << (-s));
      lo = min(lo, r);
      hi = max(hi, r);
    }
  }
  *lo_out = lo;
  *hi_out = hi;
}

template <int GROUP>
__device__ FitResult fit_range(const void* __restrict__ values, int dtype, uint64_t a, uint32_t N,
                               int model, uint32_t rank, FitShared* sm) {
  const bool lin = model == LECO_MODEL_LINEAR && N >= 2;
  const bool u32 = dtype == LECO_U32;
  const uint32_t* v32 = static_cast<const uint32_t*>(values) + a;
  const uint64_t* v64 = static_cast<const uint64_t*>(values) + a;
  i128 S;
  int64_t mx, mn;
  if (u32)
    fit_pass1<GROUP>(v32, N, lin, rank, &S, &mx, &mn);
  else
    fit_pass1<GROUP>(v64, N, lin, rank, &S, &mx, &mn);
  if (GROUP > 1) {
    S = warp_sum_i128(S);
    mx = warp_max_i64(mx);
    mn = warp_min_i64(mn);
  }
  const uint32_t lane = rank & 31u;
  FitParams P;
  if (GROUP == 1) {
    P = solve_params(S, mx, mn, N, lin);
  } else if (GROUP == 32) {
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
      const uint64_t v = u32 ? (uint64_t)__ldg(v32 + x) : __ldg(v64 + x);
      zmax = max(zmax, zz_encode((int64_t)(v - (uint64_t)P.fb_shift)));
    }
    if (GROUP > 1) zmax = warp_max_u64(zmax);
  } else {
    if (u32)
      fit_pass2<GROUP>(v32, N, P.B, P.s, rank, &lo, &hi);
    else
      fit_pass2<GROUP>(v64, N, P.B, P.s, rank, &lo, &hi);
    if (GROUP > 1) {
      lo = warp_min_i64(lo);
      hi = warp_max_i64(hi);
    }
  }
  FitResult R;
  if (GROUP == 1) {
    R = finish_fit(P, lo, hi, zmax);
  } else if (GROUP == 32) {
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
