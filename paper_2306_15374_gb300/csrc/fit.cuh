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
// values) take one native 64-bit division when |num| < 2^64 (the common case of short partitions),
// else two native 64-bit divisions and one 128-by-64 long division; wider divisors use the generic
// 128-bit routine, whose bit-serial latency would otherwise stall a whole CTA per fitted partition.
__host__ __device__ __forceinline__ i128 floordiv_i128(i128 num, i128 den) {
  if ((den >> 64) == 0 && num != ((i128)1 << 127)) {
    const uint64_t d = (uint64_t)den;
    const bool neg = num < 0;
    const u128 u = neg ? (u128)0 - (u128)num : (u128)num;
    const uint64_t hi = (uint64_t)(u >> 64), lo = (uint64_t)u;
    if (hi == 0) {
      const uint64_t q0 = lo / d, r0 = lo - q0 * d;
      return neg ? -(i128)q0 - (r0 != 0 ? 1 : 0) : (i128)q0;
    }
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
  // N (N^2 - 1) as a 64 x 64 -> 128-bit product (N^2 fits 64 bits)
  const i128 D = lin ? (i128)((u128)(uint64_t)N * ((uint64_t)N * N - 1)) : (i128)1;
  const i128 sixS = lin ? mul_i128_u64(S, 6) : (i128)0;
  const i128 a6 = sixS < 0 ? -sixS : sixS;
  // ceil(|6S| / D); without a division for the constant model (0) and for two values (D = 6: |S|)
  const i128 Q = !lin ? (i128)0 : (N == 2 ? (S < 0 ? -S : S) : floordiv_i128(a6 + D - 1, D));
  const i128 amx = mx < 0 ? -(i128)mx : (i128)mx;
  const i128 amn = mn < 0 ? -(i128)mn : (i128)mn;
  const i128 M = amx > amn ? amx : amn;
  // (Q + 1) N as a 64 x 64 -> 128-bit product; Q >= 2^62 already puts U above 2^62 (the fallback)
  const bool huge = (Q >> 62) != 0;
  const i128 U = M + ((i128)mx - (i128)mn) + (huge ? (i128)0 : (i128)((u128)(uint64_t)(Q + 1) * N)) + 4;
  const int eU = huge ? 127 : bitlen_u128((u128)U);
  if (eU > 62) {
    const i128 t = (i128)mn + (((i128)mx - (i128)mn + 1) >> 1);  // >= 1: the shift is the halving
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
  if (lin && N == 2) {  // q = S exactly: B = S 2^s, or round(S / 2^-s) half up by a shift
    B = s >= 0 ? (i128)((u128)S << s) : (2 * S + ((i128)1 << (-s))) >> (1 - s);
  } else if (lin) {
    if (s >= 0)
      B = round_half_up_i128((i128)((u128)sixS << s), D);  // sixS 2^s
    else
      B = round_half_up_i128(sixS, (i128)((u128)D << (-s)));
  }
  P.fallback = 0;
  P.s = s;
  P.B = (int64_t)B;
  P.fb_shift = 0;
  return P;
}

// step 6 alone (one thread): the width b, without the binary64 parameters (sizing only)
__device__ __forceinline__ uint32_t finish_width(const FitParams& P, int64_t lo, int64_t hi, uint64_t fb_maxzz) {
  if (P.fallback) return (uint32_t)bitlen_u64(fb_maxzz);
  const int s = P.s;
  const i128 t = (i128)lo + (((i128)hi - (i128)lo + 1) >> 1);
  const i128 shift = s >= 0 ? t : (t >> (-s)) * ((i128)1 << (-s));
  const int64_t lo2 = (int64_t)((i128)lo - shift), hi2 = (int64_t)((i128)hi - shift);
  return (uint32_t)bitlen_u64(max(zz_encode(lo2), zz_encode(hi2)));
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
  const i128 t = (i128)lo + (((i128)hi - (i128)lo + 1) >> 1);
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
// partial stays below 2^62), then folded into 128 bits. Pairs of warps on one partition (GROUP 64,
// partitions of 1024+ values) keep sixteen loads in flight per lane, other groups eight.
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
#pragma unroll (GROUP == 64 ? 16 : 8)
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
#pragma unroll 8
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
#pragma unroll (GROUP == 64 ? 16 : 8)
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

// barrier of a fitting group wider than a warp: the CTA (bar_id < 0) or named barrier bar_id over
// the group's nthreads threads (several groups in one CTA)
__device__ __forceinline__ void group_sync(int bar_id, uint32_t nthreads) {
  if (bar_id < 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthreads) : "memory");
}

template <int GROUP>
__device__ FitResult fit_range(const void* __restrict__ values, int dtype, uint64_t a, uint32_t N,
                               int model, uint32_t rank, FitShared* sm, int bar_id = -1) {
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
    group_sync(bar_id, GROUP);
    if (rank == 0) {
      for (int k = 1; k < GROUP / 32; k++) {
        S += sm->S[k];
        mx = max(mx, sm->mx[k]);
        mn = min(mn, sm->mn[k]);
      }
      sm->P = solve_params(S, mx, mn, N, lin);
    }
    group_sync(bar_id, GROUP);
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
    group_sync(bar_id, GROUP);
    if (rank == 0) {
      for (int k = 1; k < GROUP / 32; k++) {
        hi = max(hi, sm->mx[k]);
        lo = min(lo, sm->mn[k]);
        zmax = max(zmax, sm->zmax[k]);
      }
      sm->R = finish_fit(P, lo, hi, zmax);
    }
    group_sync(bar_id, GROUP);
    R = sm->R;
    group_sync(bar_id, GROUP);  // sm is reused by the next partition
  }
  return R;
}

// ------------------------------------------------------------------------------ polynomial model
//
// §3.1 names polynomial terms among the model family; §4 chooses per partition among constant,
// linear and polynomials up to degree three. This fit follows one exact reading of that choice:
//  1. one pass: min, max, and S_j = sum p_j(x) w_x (j = 1..3) over the Gram polynomials of the
//     partition, p1 = x', p2 = 3x'^2 - (N^2-1), p3 = 5x'^3 - (3N^2-7)x' with x' = 2x - (N-1); the p_j
//     are orthogonal to 1 and to each other over x < N, so S_j / |p_j|^2 is the least-squares
//     coefficient c_j of p_j for any degree that includes it (and S_1 is the line's moment);
//  2. a thread solves the constant and linear parameters (as for those models) and, when
//     64 <= N <= 16384 and max - min < 2^62, the quadratic and cubic grids: c_j as one binary64
//     division of the two integers (each converted from sign and magnitude), s_j = min(62, 61 - e_j)
//     with |c_j| < 2^e_j, S = max s_j capped so that every K_j 2^(S - s_j) p_j stays below 2^124,
//     K_j = round(c_j 2^s_j) half up;
//  3. a second pass: the linear residual range (or the fallback's widest zigzag residual) and, per
//     polynomial, the range of w_x - floor(F(x) / 2^S) (F = sum K_j 2^(S - s_j) p_j(x), exact);
//  4. a thread sizes the four candidates (256 + N b for constant and linear, 576 + N b for the
//     polynomials, whose minimax intercept T and width follow from their range as for the line) and
//     keeps the smallest, ties to the earlier.

// headroom (bits) of K_j 2^(S - s_j) p_j below 2^124: |K_j| <= 2^61, |p_j| < 2^14, 2^29, 2^43
__host__ __device__ constexpr int32_t poly_headroom(int j) { return j == 1 ? 49 : (j == 2 ? 34 : 20); }

// |p_j|^2 over N points: N(N^2-1)/3, 4N(N^2-1)(N^2-4)/5, 4N(N^2-1)(N^2-4)(N^2-9)/7
__device__ __forceinline__ i128 gram_norm(int j, uint32_t N) {
  const i128 n = N, n2 = n * n;
  const i128 base = n * (n2 - 1);
  if (j == 1) return floordiv_i128(base, 3);
  if (j == 2) return floordiv_i128(4 * base * (n2 - 4), 5);
  return floordiv_i128(4 * base * (n2 - 4) * (n2 - 9), 7);
}

// binary64 from sign and magnitude: +-(double(hi) 2^64 + double(lo)), each step rounded to nearest
__device__ __forceinline__ double i128_to_f64(i128 v) {
  const u128 mag = v < 0 ? (u128)0 - (u128)v : (u128)v;
  const double d = __dadd_rn(__dmul_rn(__ull2double_rn((uint64_t)(mag >> 64)), 18446744073709551616.0),
                             __ull2double_rn((uint64_t)mag));
  return v < 0 ? -d : d;
}

// F(x) = sum_j K_j 2^(S - s_j) p_j(x) expanded in powers of the local index x (all exact):
// p1 = 2x + (1-N), p2 = 12x^2 + (12-12N)x + (2N^2-6N+4),
// p3 = 40x^3 + (60-60N)x^2 + (24N^2-60N+44)x + (-2N^3+12N^2-22N+12).
__host__ __device__ __forceinline__ PolyAux poly_aux_from(const int64_t* K, const int32_t* sj, int32_t S, uint32_t N) {
  const i128 n = N;
  const i128 G1 = (i128)K[0] * ((i128)1 << (S - sj[0]));
  const i128 G2 = (i128)K[1] * ((i128)1 << (S - sj[1]));
  const i128 G3 = (i128)K[2] * ((i128)1 << (S - sj[2]));
  i128 a[4];
  a[3] = 40 * G3;
  a[2] = 12 * G2 + (60 - 60 * n) * G3;
  a[1] = 2 * G1 + (12 - 12 * n) * G2 + (24 * n * n - 60 * n + 44) * G3;
  a[0] = (1 - n) * G1 + (2 * n * n - 6 * n + 4) * G2 + (-2 * n * n * n + 12 * n * n - 22 * n + 12) * G3;
  PolyAux r;
  for (int k = 0; k < 4; k++) {
    r.a[k][0] = (uint64_t)(u128)a[k];
    r.a[k][1] = (uint64_t)((u128)a[k] >> 64);
  }
  return r;
}

// The cubic F(x) = c0 + c1 x + c2 x^2 + c3 x^3 (128-bit, from a PolyAux row) at x and its forward
// differences over the stride h, each multiplied by 2^up modulo 2^128:
// D1 = c1 h + c2 (2xh + h^2) + c3 (3x^2 h + 3x h^2 + h^3), D2 = c2 2h^2 + c3 (6x h^2 + 6h^3),
// D3 = c3 6h^3 (x and h below 2^14 and 2^8 keep every bracket inside 64 bits). Stepping
// F += D1, D1 += D2, D2 += D3 then gives F at x + h, x + 2h, ... exactly (modulo 2^128).
struct PolySteps {
  u128 F, D1, D2, D3;
};

__device__ __forceinline__ PolySteps poly_steps(const PolyAux& q, uint64_t x, uint64_t h, uint32_t up) {
  u128 c[4];
  for (int k = 0; k < 4; k++) c[k] = ((u128)q.a[k][1] << 64) | q.a[k][0];
  PolySteps r;
  r.F = (((c[3] * x + c[2]) * x + c[1]) * x + c[0]) << up;
  r.D1 = (c[1] * h + c[2] * (2 * x * h + h * h) + c[3] * (3 * x * x * h + 3 * x * h * h + h * h * h)) << up;
  r.D2 = (c[2] * (2 * h * h) + c[3] * (6 * x * h * h + 6 * h * h * h)) << up;
  r.D3 = (c[3] * (6 * h * h * h)) << up;
  return r;
}

__device__ __forceinline__ void poly_step(PolySteps& r) {
  r.F += r.D1;
  r.D1 += r.D2;
  r.D2 += r.D3;
}

// one polynomial candidate's grid (step 2)
struct PolyGrid {
  int64_t K[3];
  int32_t sj[3];
  int32_t S;
  int32_t valid;
};

__device__ PolyGrid poly_grid(const i128* Sm, uint32_t N, int degree) {
  PolyGrid g;
  g.valid = 0;
  g.S = 0;
  double c[3] = {0.0, 0.0, 0.0};
  int32_t cap = 1 << 30;
  for (int j = 0; j < 3; j++) {
    g.K[j] = 0;
    g.sj[j] = 0;
  }
  for (int j = 0; j < degree; j++) {
    c[j] = __ddiv_rn(i128_to_f64(Sm[j]), i128_to_f64(gram_norm(j + 1, N)));
    if (c[j] != 0.0) {
      int e;
      frexp(c[j], &e);  // |c| < 2^e
      int32_t sj = 61 - e;
      if (sj > 62) sj = 62;
      if (sj < 0) return g;
      g.sj[j] = sj;
      g.S = max(g.S, sj);
      cap = min(cap, sj + poly_headroom(j + 1));
    }
  }
  g.S = min(g.S, cap);
  for (int j = 0; j < degree; j++) {
    g.sj[j] = min(g.sj[j], g.S);
    const double y = __dmul_rn(c[j], pow2(g.sj[j]));  // exact: a power-of-two scale
    const double f = floor(y);
    g.K[j] = __double2ll_rz(f) + (__dsub_rn(y, f) >= 0.5 ? 1 : 0);
  }
  g.valid = 1;
  return g;
}

// What the polynomial model chose for one partition: kind 0 constant, 1 linear (R: the record's
// theta, s and b exactly as those models write them), 2 quadratic, 3 cubic (pc: its block).
struct FitChoice {
  FitResult R;
  PolyCoef pc;
  uint32_t kind;
  uint32_t b;
};

// The polynomial model's fit runs as four phases, each its own kernel so that none carries the
// others' registers: moments (a warp per partition), plan (a thread: every candidate's parameters),
// ranges (a warp: the residual ranges under them), choice (a thread: sizes and the record).

// phase 1 result: min, max and the Gram moments S_j = sum p_j(x) w_x (S_1 is the line's moment)
struct PolyMom {
  i128 S[3];
  int64_t mx, mn;
};
static_assert(sizeof(PolyMom) == 64, "poly moments layout");

// phase 2 result
struct PolyPlan {
  FitParams PC, PL;  // constant and linear parameters (as those models solve them)
  PolyGrid G[2];     // quadratic and cubic grids (valid = 0: the candidate does not apply)
  PolyAux Q[2];      // their F as 128-bit monomial coefficients
  int32_t fast[2];   // |floor(F / 2^S)| is bounded so that every residual fits int64 (see poly_plan)
  int32_t pad[2];
};

// phase 3 result
struct PolyRange {
  int64_t lo, hi;   // the line's residual range (not fallback)
  uint64_t zmax;    // the fallback's widest zigzag residual
  int64_t plo[2], phi[2];
  int32_t bad[2];   // a residual outside int64: the candidate does not apply
};

__device__ __forceinline__ int64_t poly_value_at(const uint32_t* v32, const uint64_t* v64, bool u32, uint32_t x) {
  return u32 ? (int64_t)__ldg(v32 + x) : (int64_t)__ldg(v64 + x);
}

// phase 1 by one warp; the result in lane 0
__device__ PolyMom poly_moments_warp(const void* __restrict__ values, int dtype, uint64_t a, uint32_t N,
                                     uint32_t lane) {
  const bool u32 = dtype == LECO_U32;
  const uint32_t* v32 = static_cast<const uint32_t*>(values) + a;
  const uint64_t* v64 = static_cast<const uint64_t*>(values) + a;
  const bool poly_len = N >= kPolyMinLen && N <= kPolyMaxLen;
  int64_t mx = INT64_MIN, mn = INT64_MAX;
  i128 Sm[3] = {0, 0, 0};
  const int64_t nm1 = (int64_t)N - 1;
  const int64_t n2m1 = (int64_t)N * N - 1, c3 = 3 * (int64_t)N * N - 7;
  for (uint32_t x = lane; x < N; x += 32) {
    const int64_t w = poly_value_at(v32, v64, u32, x);
    mx = max(mx, w);
    mn = min(mn, w);
    const int64_t xp = 2 * (int64_t)x - nm1;
    Sm[0] += (i128)xp * w;
    if (poly_len) {
      const int64_t xp2 = xp * xp;
      Sm[1] += (i128)(3 * xp2 - n2m1) * w;
      Sm[2] += (i128)((5 * xp2 - c3) * xp) * w;
    }
  }
  PolyMom M;
  for (int j = 0; j < 3; j++) M.S[j] = warp_sum_i128(Sm[j]);
  M.mx = warp_max_i64(mx);
  M.mn = warp_min_i64(mn);
  return M;
}

// phase 2 (one thread)
__device__ PolyPlan poly_plan(const PolyMom& M, uint32_t N) {
  PolyPlan P;
  P.PC = solve_params(M.S[0], M.mx, M.mn, N, false);
  P.PL = solve_params(M.S[0], M.mx, M.mn, N, N >= 2);
  const bool elig = N >= kPolyMinLen && N <= kPolyMaxLen && (i128)M.mx - (i128)M.mn < ((i128)1 << 62);
  for (int d = 0; d < 2; d++) {
    P.G[d].valid = 0;
    P.fast[d] = 0;
    if (elig) P.G[d] = poly_grid(M.S, N, 2 + d);
    if (!P.G[d].valid) continue;
    P.Q[d] = poly_aux_from(P.G[d].K, P.G[d].sj, P.G[d].S, N);
    // |F(x)| <= sum_j |K_j| 2^(S - s_j) max|p_j| with max|p_1| < N, max|p_2| <= 2N^2, max|p_3| <= 2N^3;
    // with q = floor(F / 2^S) in [-Bq, Bq], every residual w - q lies in [mn - Bq, mx + Bq]
    const u128 n = N;
    const u128 bnd[3] = {n, 2 * n * n, 2 * n * n * n};
    u128 Fb = 0;
    for (int j = 0; j < 3; j++) {
      const int64_t k = P.G[d].K[j];
      const u128 ak = (u128)(k < 0 ? -(i128)k : (i128)k) << (P.G[d].S - P.G[d].sj[j]);
      Fb += ak * bnd[j];
    }
    const i128 Bq = (i128)(Fb >> P.G[d].S) + 1;
    P.fast[d] = Bq < ((i128)1 << 62) && (i128)M.mn - Bq > (i128)INT64_MIN && (i128)M.mx + Bq < (i128)INT64_MAX;
  }
  return P;
}

// phase 3 by one warp; the result in lane 0. One pass: the line's residual (or the fallback's
// zigzag residual) and both polynomials' residuals at the lane's positions x = lane + 32k, each
// polynomial's F by forward differences over the stride 32 (exact 128-bit; x < 2^14, so every
// bracket fits 64 bits).
__device__ PolyRange poly_ranges_warp(const void* __restrict__ values, int dtype, uint64_t a, uint32_t N,
                                      uint32_t lane, const PolyPlan* __restrict__ plan) {
  const bool u32 = dtype == LECO_U32;
  const uint32_t* v32 = static_cast<const uint32_t*>(values) + a;
  const uint64_t* v64 = static_cast<const uint64_t*>(values) + a;
  const int64_t B = plan->PL.B, fb = plan->PL.fb_shift;
  const int32_t s = plan->PL.s, fallback = plan->PL.fallback;
  bool valid[2], fast[2];
  int32_t S[2];
  PolySteps Fd[2];
  for (int d = 0; d < 2; d++) {
    valid[d] = plan->G[d].valid != 0;
    fast[d] = valid[d] && plan->fast[d];
    S[d] = plan->G[d].S;
    // fast: carried times 2^(64-S) modulo 2^128, so that floor(F / 2^S) mod 2^64 (= floor(F / 2^S),
    // which the plan bounded inside int64) is the high half
    const uint32_t up = fast[d] ? 64u - (uint32_t)S[d] : 0u;
    Fd[d] = valid[d] ? poly_steps(plan->Q[d], lane, 32, up) : PolySteps{0, 0, 0, 0};
  }
  PolyRange R;
  int64_t lo = INT64_MAX, hi = INT64_MIN;
  uint64_t zmax = 0;
  int64_t plo[2] = {INT64_MAX, INT64_MAX}, phi[2] = {INT64_MIN, INT64_MIN};
  int bad[2] = {0, 0};
  for (uint32_t x = lane; x < N; x += 32) {
    const int64_t w = poly_value_at(v32, v64, u32, x);
    if (fallback) {
      zmax = max(zmax, zz_encode((int64_t)((uint64_t)w - (uint64_t)fb)));
    } else {
      const uint64_t Fl = (uint64_t)B * x;
      const int64_t r = w - (s >= 0 ? ((int64_t)Fl >> s) : (int64_t)(Fl << (-s)));
      lo = min(lo, r);
      hi = max(hi, r);
    }
#pragma unroll
    for (int d = 0; d < 2; d++) {
      if (!valid[d]) continue;
      if (fast[d]) {
        const int64_t r = w - (int64_t)(uint64_t)(Fd[d].F >> 64);
        plo[d] = min(plo[d], r);
        phi[d] = max(phi[d], r);
      } else {
        const i128 r = (i128)w - ((i128)Fd[d].F >> S[d]);
        if (r > (i128)INT64_MAX || r < (i128)INT64_MIN) {
          bad[d] = 1;
        } else {
          plo[d] = min(plo[d], (int64_t)r);
          phi[d] = max(phi[d], (int64_t)r);
        }
      }
      poly_step(Fd[d]);
    }
  }
  R.lo = warp_min_i64(lo);
  R.hi = warp_max_i64(hi);
  R.zmax = warp_max_u64(zmax);
  for (int d = 0; d < 2; d++) {
    R.plo[d] = warp_min_i64(plo[d]);
    R.phi[d] = warp_max_i64(phi[d]);
    R.bad[d] = __any_sync(0xffffffffu, bad[d]);
  }
  return R;
}

// phase 4 (one thread): size the four candidates (256 + N b for constant and linear, 576 + N b for
// the polynomials, whose minimax intercept and width follow from their range as for the line) and
// keep the smallest, ties to the earlier
__device__ FitChoice poly_choose(const PolyMom& M, const PolyPlan& P, const PolyRange& R, uint32_t N) {
  FitChoice C;
  C.R = finish_fit(P.PC, M.mn, M.mx, R.zmax);  // a constant fallback implies the linear one: same zmax
  C.kind = 0;
  C.b = C.R.b;
  uint64_t best = kSmBits + (uint64_t)N * C.R.b;
  const FitResult RL = finish_fit(P.PL, R.lo, R.hi, R.zmax);
  if (kSmBits + (uint64_t)N * RL.b < best) {
    best = kSmBits + (uint64_t)N * RL.b;
    C.R = RL;
    C.kind = 1;
    C.b = RL.b;
  }
  for (int d = 0; d < 2; d++) {
    if (!P.G[d].valid || R.bad[d]) continue;
    const i128 t = (i128)R.plo[d] + (((i128)R.phi[d] - (i128)R.plo[d] + 1) >> 1);
    const uint64_t z = max(zz_encode((int64_t)((i128)R.plo[d] - t)), zz_encode((int64_t)((i128)R.phi[d] - t)));
    const uint32_t b = (uint32_t)bitlen_u64(z);
    const uint64_t size = kSmBits + kPolyBlockBits + (uint64_t)N * b;
    if (size < best) {
      best = size;
      C.kind = 2 + d;
      C.b = b;
      C.pc.T = (int64_t)t;
      for (int j = 0; j < 3; j++) C.pc.K[j] = P.G[d].K[j];
      C.pc.E = (uint64_t)P.G[d].sj[0] | ((uint64_t)P.G[d].sj[1] << 8) | ((uint64_t)P.G[d].sj[2] << 16);
    }
  }
  return C;
}

}  // namespace
}  // namespace leco
