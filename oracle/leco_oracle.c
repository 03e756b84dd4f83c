/*
 * LeCo CPU oracle — plain, slow, obviously correct C for what the GPU path computes.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link, load or call this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg use it. It shares
 * no code, header, table or constant generator with the CUDA library; the byte format below is
 * restated here from the format definition, not included.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared (no FMA contraction:
 * the model prediction is one IEEE binary64 rounding per operation).
 *
 * Paper sections followed (Liu, Zeng & Zhang, "LeCo: Lightweight Compression via Learning
 * Serial Correlations"):
 *   §3 (problem statement)   size = sum over partitions of model size + len * max delta bits
 *   §3.1 (Regressor)         least-squares line, bit-packed deltas sized by the maximum error,
 *                            minimax objective (the intercept recentering below)
 *   §3.2.1                   fixed-length partitions: partition j holds positions [jL, (j+1)L)
 *   §3.2.2                   variable-length split (cost C <= tau*S_M, the delta-tilde metric)
 *                            and merge (accept when the merged size is smaller)
 *   §3.3 (Encoder/Decoder)   header (theta0, theta1, b, start), point decode
 *                            floor(theta0 + theta1*i') + delta_{i'} from bits [b*i', b*(i'+1))
 *   §2                       FOR / RLE / Delta as special cases of the model family
 *
 * Readings where the paper is silent or garbled (each one is also listed in the design notes):
 *   R1 width: b = bitlen(max zigzag residual) = ceil(log2(max zz + 1)) (the paper's
 *      ceil(log2 |delta|) has no sign bit and gives 0 bits for |delta| = 1).
 *   R2 prediction: pred(i') = clamp_floor(fl(fl(theta1 * i') + theta0)), binary64, one rounding
 *      per operation; clamp_floor(NaN) = 0, >= 2^63 -> INT64_MAX, < -2^63 -> INT64_MIN.
 *   R3 value = (pred + unzigzag(field)) mod 2^64; for 32-bit columns truncated to 32 bits.
 *   R4 the fit treats a 64-bit value as its two's complement int64 (w = (int64)v).
 *   R5 linear fit: exact rational least-squares slope q = 6S/D, S = sum (2x-(N-1))(w_x - w_0),
 *      D = N(N^2-1); the slope is snapped to the grid 2^-s (round half up), the intercept is the
 *      minimax one for that slope (recentering); s comes from the magnitude bound U below.
 *   R6 format: LSB-first bit stream of 64-bit little-endian words, dense offsets, >= 2 zero
 *      padding words, total rounded up to 16 bytes; 32-byte records
 *      {theta0 f64, theta1 f64, start u64, word3 = off:48 | b:7 | s:7 | exact:1 | 0:1}.
 *   R7 var split: one left-to-right sweep per chunk (chunk edges always cut), delta-tilde =
 *      bitlen(max d - min d) over the inner differences, S_M = 256 bits (one record).
 *   R8 var merge: (seq) the paper's left-to-right passes; (round) all pairs whose gain is a local
 *      maximum merged at once per round, equal gains ordered by a SplitMix64 hash of the position.
 *   R9 partition-size search (§3.2.1): samples are k = max(1, floor(frac n / N)) subsequences of
 *      length N starting at SplitMix64(seed + i) mod (n - N + 1); sizes of fixed partitions cut from
 *      each subsequence's start; exponential phase over powers of two that ends after the first size
 *      above its predecessor's; back search probing best +- step (step from half the best L,
 *      halved when neither probe is smaller); stop when the step is 0 or a move gains < 0.01 %.
 *  R10 polynomial model (§3.1 lists polynomial terms; §4 compares constant, linear and polynomials
 *      up to degree three, choosing per partition): with model 2 each partition takes the smallest
 *      of four candidates by exact size S + len * b, ties to the earlier one: constant (R5 with
 *      q = 0), linear (R5), quadratic, cubic (S = 256 bits for the first two; 576 for the
 *      polynomials, whose five 64-bit words sit in the stream ahead of the residuals).
 *      A polynomial of degree d in {2, 3} is fitted on the discrete orthogonal polynomials of the
 *      partition, x' = 2x - (N-1): p1 = x', p2 = 3x'^2 - (N^2-1), p3 = 5x'^3 - (3N^2-7)x'.
 *      Least squares gives c_j = S_j / |p_j|^2 with the exact integer S_j = sum p_j(x)(w_x - w_0);
 *      c_j is one binary64 division of the two integers, each converted from sign and magnitude
 *      as +-(double(hi) * 2^64 + double(lo)). Each coefficient has its own grid: sj = min(62, 61 - e)
 *      with |c_j| < 2^e, K_j = round(c_j 2^sj) (half up), sj < 0 rejects the candidate; S = max sj,
 *      capped so that every term K_j 2^(S - sj) p_j(x) stays below 2^124 (the finer grids are
 *      coarsened to the cap). Prediction pred(x) = T + floor(F(x) / 2^S) mod 2^64 with
 *      F = sum K_j 2^(S - sj) p_j(x) (an exact integer, no floating point), T the minimax intercept
 *      of the residuals w - floor(F / 2^S). A candidate needs 64 <= N <= 16384,
 *      max w - min w < 2^62 and every such residual inside int64. Record: theta0 = theta1 = 0,
 *      word3 bit 63 set, exact bit 0, s = 0; stream at off: T, K1, K2, K3 (64 bits each, K3 = 0
 *      for the quadratic), the exponent word s1 | s2 << 8 | s3 << 16, then residual k at
 *      off + 320 + b k. Variable partitioning and the size search keep the linear size (§3.2).
 *  R11 seeded split (§3.2.2, selecting good starting positions: for a degree-k regressor, start
 *      where the (k+1)-th order deltas are smallest): each chunk has one seed, the first window of
 *      three values whose second-order delta has the shortest zigzag code; partitions grow from it
 *      to the right with the greedy rule and, with the same rule on the values read backwards, to
 *      the left; the seed and the chunk edge are cuts. (One seed per chunk: the paper's precedence
 *      among seeds growing into each other does not arise.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define ORC_MODEL_CONSTANT 0
#define ORC_MODEL_LINEAR 1
#define ORC_MODEL_POLY 2

/* One 32-byte partition header (§3.3 storage format, with this format's offset/grid fields). */
typedef struct {
  double theta0;
  double theta1;
  uint64_t start;
  uint64_t word3;
} orc_record;

/* Everything the regressor decides for one partition (exposed for the pins). */
typedef struct {
  double theta0, theta1;
  int64_t A, B;      /* grid intercept/slope: theta0 = A*2^-s (s>=0) or A*2^|s| (s<0); same for B */
  int32_t s;         /* grid exponent */
  int32_t exact;     /* 1: the integer formula equals the binary64 prediction for every x < N */
  int32_t b;         /* residual width in bits, 0..64 */
  int32_t fallback;  /* 1: magnitude bound too large; constant model on the 2^11 grid */
  int64_t shift;     /* recentering shift applied to the zero-intercept residuals */
} orc_fit;

/* ---------------------------------------------------------------- small helpers */

static void orc_die(const char* why) {
  (void)why;
  abort(); /* an oracle invariant failed: the reasoning in the header is wrong, not the input */
}

static int bitlen_u128(u128 x) {
  int n = 0;
  while (x) {
    n++;
    x >>= 1;
  }
  return n;
}

static int bitlen_u64(uint64_t x) { return bitlen_u128((u128)x); }

static i128 abs128(i128 x) { return x < 0 ? -x : x; }

/* zigzag: 0,-1,1,-2,2,... -> 0,1,2,3,4,... (residual sign folded into the low bit, R1) */
static uint64_t zigzag64(int64_t r) { return ((uint64_t)r << 1) ^ (uint64_t)(r >> 63); }

static int64_t unzigzag64(uint64_t z) { return (int64_t)((z >> 1) ^ (0 - (z & 1))); }

/* mathematical floor division, den > 0 */
static i128 floordiv128(i128 num, i128 den) {
  i128 q = num / den;
  if ((num % den) != 0 && num < 0) q -= 1;
  return q;
}

/* round num/den half up = floor((2 num + den) / (2 den)), den > 0 (R5) */
static i128 round_half_up128(i128 num, i128 den) { return floordiv128(2 * num + den, 2 * den); }

/* ------------------------------------------------------------ prediction (§3.3, R2) */

int64_t orc_clamp_floor(double y) {
  if (isnan(y)) return 0;
  if (y >= 9223372036854775808.0) return INT64_MAX;
  if (y < -9223372036854775808.0) return INT64_MIN;
  return (int64_t)floor(y);
}

/* pred(i') = clamp_floor(fl(fl(theta1 * i') + theta0)); compiled without FMA contraction. */
int64_t orc_predict(double theta0, double theta1, uint64_t x) {
  double xd = (double)x;
  volatile double prod = theta1 * xd; /* one rounding */
  volatile double sum = prod + theta0;  /* one rounding */
  return orc_clamp_floor(sum);
}

/* ------------------------------------------------------------ regressor (§3.1, R4, R5) */

/*
 * Fit one partition of N >= 1 values with the constant (FOR) or linear model.
 * Steps, in order:
 *  1. least-squares slope q = 6S/D as an exact rational (0 for the constant model or N = 1);
 *  2. magnitude bound U = M + (Wmax - Wmin) + (ceil|q| + 1) N + 4, M = max |w|;
 *     if bitlen(U) > 62 the partition falls back to the constant model on the grid 2^11
 *     (theta0 = the midrange rounded down to a multiple of 2048, residuals mod 2^64);
 *  3. grid exponent s = min(52, 52 - bitlen(U)); slope B = round(q 2^s);
 *  4. zero-intercept residuals r0_x = w_x - floor(B x 2^-s), lo = min, hi = max;
 *  5. minimax recentering: t = lo + ceil((hi-lo)/2), rounded down to the grid step 2^max(0,-s);
 *  6. residual r_x = r0_x - shift, width b = bitlen(max zigzag(r_x)).
 */
void orc_fit_partition(const uint64_t* v, uint64_t N, int model, orc_fit* out) {
  memset(out, 0, sizeof(*out));
  if (model != ORC_MODEL_CONSTANT && model != ORC_MODEL_LINEAR) orc_die("model");
  if (N == 0) orc_die("empty partition");
  if (N > ((uint64_t)1 << 24)) orc_die("partition longer than 2^24");

  /* w = two's complement view of the value (R4) */
  i128 w0 = (int64_t)v[0];
  i128 wmax = w0, wmin = w0;
  for (uint64_t x = 0; x < N; x++) {
    i128 w = (int64_t)v[x];
    if (w > wmax) wmax = w;
    if (w < wmin) wmin = w;
  }

  /* step 1: S = sum (2x - (N-1)) (w_x - w_0), D = N (N^2 - 1) */
  i128 S = 0, D = 1;
  if (model == ORC_MODEL_LINEAR && N >= 2) {
    for (uint64_t x = 0; x < N; x++) {
      i128 u = (i128)(2 * (int64_t)x) - (i128)(N - 1);
      i128 y = (i128)(int64_t)v[x] - w0;
      S += u * y;
    }
    D = (i128)N * ((i128)N * (i128)N - 1);
  }
  i128 sixS = 6 * S;

  /* step 2: magnitude bound */
  i128 Q = floordiv128(abs128(sixS) + D - 1, D); /* ceil(|q|) */
  i128 M = abs128(wmax) > abs128(wmin) ? abs128(wmax) : abs128(wmin);
  i128 U = M + (wmax - wmin) + (Q + 1) * (i128)N + 4;
  int eU = bitlen_u128((u128)U);

  int64_t* r0 = (int64_t*)malloc(sizeof(int64_t) * N);
  if (!r0) orc_die("oom");

  if (eU > 62) {
    /* fallback: constant model on the 2^11 grid (always exact: |theta0| <= 2^63 - 2^11),
       residuals taken mod 2^64 */
    i128 t = wmin + (wmax - wmin + 1) / 2;
    i128 tg = floordiv128(t, (i128)1 << 11);
    out->fallback = 1;
    out->exact = 1;
    out->s = -11;
    out->A = (int64_t)tg;
    out->B = 0;
    out->shift = (int64_t)(tg * 2048);
    out->theta0 = ldexp((double)(int64_t)tg, 11);
    out->theta1 = 0.0;
    uint64_t maxzz = 0;
    for (uint64_t x = 0; x < N; x++) {
      uint64_t z = zigzag64((int64_t)(v[x] - (uint64_t)out->shift));
      if (z > maxzz) maxzz = z;
    }
    out->b = bitlen_u64(maxzz);
    free(r0);
    return;
  }

  /* step 3: grid exponent and slope */
  int s = 52 - eU;
  if (s > 52) s = 52;
  i128 B;
  if (model != ORC_MODEL_LINEAR || N < 2) {
    B = 0;
  } else if (s >= 0) {
    B = round_half_up128(sixS * ((i128)1 << s), D);
  } else {
    B = round_half_up128(sixS, D * ((i128)1 << (-s)));
  }

  /* step 4: zero-intercept residuals */
  i128 lo = 0, hi = 0;
  for (uint64_t x = 0; x < N; x++) {
    i128 bx = B * (i128)x;
    i128 line = s >= 0 ? floordiv128(bx, (i128)1 << s) : bx * ((i128)1 << (-s));
    i128 r = (i128)(int64_t)v[x] - line;
    if (x == 0 || r < lo) lo = r;
    if (x == 0 || r > hi) hi = r;
    if (r > INT64_MAX || r < INT64_MIN) orc_die("residual beyond int64");
    r0[x] = (int64_t)r;
  }

  /* step 5: minimax recentering on the grid */
  i128 t = lo + (hi - lo + 1) / 2; /* lo + ceil((hi-lo)/2), hi >= lo */
  i128 g = s >= 0 ? 1 : ((i128)1 << (-s));
  i128 tg = floordiv128(t, g);
  i128 shift = tg * g;
  i128 A = s >= 0 ? shift * ((i128)1 << s) : tg;

  /* invariants that make the integer formula equal the binary64 definition (checked, not assumed) */
  for (int e = 0; e < 2; e++) {
    i128 x = e == 0 ? 0 : (i128)(N - 1);
    i128 f = A + B * x;
    i128 bx = B * x;
    i128 lim = (i128)1 << 53;
    if (abs128(f) >= lim || abs128(bx) >= lim) orc_die("grid bound violated");
    if (s < 0 && abs128(f * ((i128)1 << (-s))) >= ((i128)1 << 63)) orc_die("int64 bound violated");
    (void)bx;
  }

  out->s = s;
  out->A = (int64_t)A;
  out->B = (int64_t)B;
  out->shift = (int64_t)shift;
  out->exact = 1;
  out->theta0 = ldexp((double)(int64_t)A, -s); /* exact: |A| < 2^53 */
  out->theta1 = ldexp((double)(int64_t)B, -s); /* exact: |B| < 2^53 */

  /* step 6: width from every residual */
  uint64_t maxzz = 0;
  for (uint64_t x = 0; x < N; x++) {
    i128 r = (i128)r0[x] - shift;
    if (r > INT64_MAX || r < INT64_MIN) orc_die("residual beyond int64");
    uint64_t z = zigzag64((int64_t)r);
    if (z > maxzz) maxzz = z;
  }
  out->b = bitlen_u64(maxzz);
  free(r0);
}

/* ------------------------------------------------------------ polynomial model (§3.1, §4, R10) */

#define ORC_POLY_MIN_LEN 64
#define ORC_POLY_MAX_LEN 16384

/* Gram polynomial p_j (j = 1, 2, 3) of N points at x, on x' = 2x - (N-1) (R10). */
i128 orc_gram_p(int j, uint64_t N, uint64_t x) {
  i128 xp = (i128)(2 * (int64_t)x) - (i128)(N - 1);
  i128 n2 = (i128)N * (i128)N;
  if (j == 1) return xp;
  if (j == 2) return 3 * xp * xp - (n2 - 1);
  if (j == 3) return 5 * xp * xp * xp - (3 * n2 - 7) * xp;
  orc_die("gram polynomial degree");
  return 0;
}

/* |p_j|^2 = sum over x < N of p_j(x)^2, closed forms (R10) */
i128 orc_gram_norm(int j, uint64_t N) {
  i128 n = (i128)N, n2 = n * n;
  if (j == 1) return n * (n2 - 1) / 3;
  if (j == 2) return 4 * n * (n2 - 1) * (n2 - 4) / 5;
  if (j == 3) return 4 * n * (n2 - 1) * (n2 - 4) * (n2 - 9) / 7;
  orc_die("gram polynomial degree");
  return 0;
}

/* integer to binary64 from sign and magnitude: +-(double(hi) * 2^64 + double(lo)) with hi, lo the
   halves of |v| (each conversion and the sum rounded to nearest: the same on every host) */
static double i128_to_double(i128 v) {
  u128 mag = v < 0 ? (u128)0 - (u128)v : (u128)v;
  double d = (double)(uint64_t)(mag >> 64) * 18446744073709551616.0 + (double)(uint64_t)mag;
  return v < 0 ? -d : d;
}

/* Everything one polynomial candidate decides (exposed for the pins). */
typedef struct {
  double c[4];      /* c[1..3]: least-squares coefficients on p_1..p_3 (c[3] = 0 for degree 2) */
  int64_t K[4];     /* K[1..3]: grid coefficients, c_j ~ K_j 2^-sj[j] */
  int32_t sj[4];    /* sj[1..3]: each coefficient's grid exponent, 0..62 */
  int64_t T;        /* minimax intercept */
  int32_t S;        /* max sj: F is evaluated on the grid 2^-S */
  int32_t b;        /* residual width */
  int32_t valid;    /* 0: the candidate does not apply (R10 conditions) */
  int32_t degree;
  uint64_t size;    /* 576 + N b when valid */
} orc_poly_fit;

/* bits a term K_j 2^(S - sj) p_j may be shifted by and stay below 2^124: |K_j| <= 2^61 and, for
   N <= 16384, |p_1| < 2^14, |p_2| < 2^29, |p_3| < 2^43 */
static const int32_t poly_headroom[4] = {0, 49, 34, 20};

/* floor(sum_j K_j p_j(x) 2^-sj / 1) = floor(F(x) / 2^S), F = sum_j K_j 2^(S - sj) p_j(x) */
static i128 poly_line(const int64_t* K, const int32_t* sj, int32_t S, uint64_t N, uint64_t x) {
  i128 F = 0;
  for (int j = 1; j <= 3; j++) F += (i128)K[j] * ((i128)1 << (S - sj[j])) * orc_gram_p(j, N, x);
  return floordiv128(F, (i128)1 << S);
}

/*
 * One polynomial candidate of degree 2 or 3 (R10), steps in order:
 *  1. applicability: 64 <= N <= 16384 and max w - min w < 2^62;
 *  2. exact moments S_j = sum p_j(x) (w_x - w_0) and least-squares coefficients c_j = S_j / |p_j|^2;
 *  3. grid exponents: sj = min(62, 61 - e_j) with |c_j| < 2^e_j (0 when c_j = 0; a negative one
 *     rejects the candidate), S = min(max sj, min over nonzero c_j of sj + headroom_j), each sj
 *     lowered to at most S, and K_j = round(c_j 2^sj) (half up);
 *  4. residuals r0_x = w_x - floor(F(x) / 2^S) (all inside int64), lo = min, hi = max;
 *  5. minimax intercept T = lo + ceil((hi - lo) / 2), width b = bitlen(max zigzag(r0 - T)).
 */
void orc_fit_poly(const uint64_t* v, uint64_t N, int degree, orc_poly_fit* out) {
  memset(out, 0, sizeof(*out));
  out->degree = degree;
  if (degree < 2 || degree > 3) orc_die("polynomial degree");
  if (N < ORC_POLY_MIN_LEN || N > ORC_POLY_MAX_LEN) return;
  i128 w0 = (int64_t)v[0], wmax = w0, wmin = w0;
  for (uint64_t x = 0; x < N; x++) {
    i128 w = (int64_t)v[x];
    if (w > wmax) wmax = w;
    if (w < wmin) wmin = w;
  }
  if (wmax - wmin >= ((i128)1 << 62)) return;

  int32_t S = 0, cap = INT32_MAX;
  for (int j = 1; j <= degree; j++) {
    i128 Sj = 0;
    for (uint64_t x = 0; x < N; x++) Sj += orc_gram_p(j, N, x) * ((i128)(int64_t)v[x] - w0);
    out->c[j] = i128_to_double(Sj) / i128_to_double(orc_gram_norm(j, N));
    if (out->c[j] != 0.0) {
      int e;
      frexp(out->c[j], &e); /* |c| < 2^e */
      int sj = 61 - e;
      if (sj > 62) sj = 62;
      if (sj < 0) return;
      out->sj[j] = sj;
      if (sj > S) S = sj;
      if (sj + poly_headroom[j] < cap) cap = sj + poly_headroom[j];
    }
  }
  if (S > cap) S = cap;
  out->S = S;
  for (int j = 1; j <= degree; j++) {
    if (out->sj[j] > S) out->sj[j] = S;
    double y = ldexp(out->c[j], out->sj[j]); /* exact: a power-of-two scale */
    double f = floor(y);
    out->K[j] = (int64_t)f + (y - f >= 0.5 ? 1 : 0);
  }

  i128 lo = 0, hi = 0;
  for (uint64_t x = 0; x < N; x++) {
    i128 r = (i128)(int64_t)v[x] - poly_line(out->K, out->sj, S, N, x);
    if (r > INT64_MAX || r < INT64_MIN) return;
    if (x == 0 || r < lo) lo = r;
    if (x == 0 || r > hi) hi = r;
  }
  i128 t = lo + (hi - lo + 1) / 2;
  uint64_t z1 = zigzag64((int64_t)(lo - t)), z2 = zigzag64((int64_t)(hi - t));
  out->T = (int64_t)t;
  out->b = bitlen_u64(z1 > z2 ? z1 : z2);
  out->valid = 1;
  out->size = 576 + N * (uint64_t)out->b;
}

/* The candidate a partition takes under model 2 (R10). */
typedef struct {
  int32_t kind; /* 0 constant, 1 linear, 2 quadratic, 3 cubic */
  int32_t pad;
  uint64_t size;
  orc_fit fit;       /* kinds 0, 1 */
  orc_poly_fit poly; /* kinds 2, 3 */
} orc_choice;

void orc_choose_model(const uint64_t* v, uint64_t N, orc_choice* out) {
  memset(out, 0, sizeof(*out));
  orc_fit f;
  orc_fit_partition(v, N, ORC_MODEL_CONSTANT, &f);
  out->kind = 0;
  out->fit = f;
  out->size = 256 + N * (uint64_t)f.b;
  orc_fit_partition(v, N, ORC_MODEL_LINEAR, &f);
  if (256 + N * (uint64_t)f.b < out->size) {
    out->kind = 1;
    out->fit = f;
    out->size = 256 + N * (uint64_t)f.b;
  }
  for (int d = 2; d <= 3; d++) {
    orc_poly_fit q;
    orc_fit_poly(v, N, d, &q);
    if (q.valid && q.size < out->size) {
      out->kind = d;
      out->poly = q;
      out->size = q.size;
    }
  }
}

/* ctypes helpers for the pins: 128-bit results as two 64-bit halves, the choice as kind + size */
void orc_gram_p_parts(int j, uint64_t N, uint64_t x, uint64_t* lo, int64_t* hi) {
  i128 v = orc_gram_p(j, N, x);
  *lo = (uint64_t)v;
  *hi = (int64_t)(v >> 64);
}
void orc_gram_norm_parts(int j, uint64_t N, uint64_t* lo, int64_t* hi) {
  i128 v = orc_gram_norm(j, N);
  *lo = (uint64_t)v;
  *hi = (int64_t)(v >> 64);
}
int orc_choose_kind(const uint64_t* v, uint64_t N, uint64_t* size) {
  orc_choice c;
  orc_choose_model(v, N, &c);
  *size = c.size;
  return c.kind;
}

/* Total bits of one partition under the model: the §3 size term S_M + len * b with S_M = 256
   (model 2: the chosen candidate's size, R10). */
uint64_t orc_partition_size_bits(const uint64_t* v, uint64_t N, int model) {
  if (model == ORC_MODEL_POLY) {
    orc_choice c;
    orc_choose_model(v, N, &c);
    return c.size;
  }
  orc_fit f;
  orc_fit_partition(v, N, model, &f);
  return 256 + N * (uint64_t)f.b;
}

/* ------------------------------------------------------------ encoder (§3.3, R6) */

static uint64_t make_word3(uint64_t off, int b, int s, int exact) {
  return (off & (((uint64_t)1 << 48) - 1)) | ((uint64_t)(b & 0x7F) << 48) |
         ((uint64_t)(s & 0x7F) << 55) | ((uint64_t)(exact & 1) << 62);
}

/* write the low b bits of field at absolute bit position pos (LSB-first) */
static void put_field(uint64_t* words, uint64_t pos, int b, uint64_t field) {
  for (int k = 0; k < b; k++) {
    if ((field >> k) & 1) {
      uint64_t p = pos + (uint64_t)k;
      words[p / 64] |= (uint64_t)1 << (p % 64);
    }
  }
}

/* bits [pos, pos+b) as an integer, LSB-first */
static uint64_t get_field(const uint64_t* words, uint64_t pos, int b) {
  uint64_t f = 0;
  for (int k = 0; k < b; k++) {
    uint64_t p = pos + (uint64_t)k;
    f |= ((words[p / 64] >> (p % 64)) & 1) << k;
  }
  return f;
}

/* words the stream needs for total_bits: ceil(bits/64) + 2 padding, rounded up to even */
uint64_t orc_words_for_bits(uint64_t total_bits) {
  uint64_t w = (total_bits + 63) / 64 + 2;
  return (w + 1) & ~(uint64_t)1;
}

/*
 * Fit every partition [starts[p], starts[p+1]) and pack the residuals (§3.3 Encoder).
 * First pass fits (model 2: chooses, R10) and sums each partition's stream bits into the offsets;
 * the second packs. Returns the padded word count, or 0 when cap_words is too small (words[] is not
 * touched then). records needs m entries.
 */
uint64_t orc_encode(const uint64_t* v, uint64_t n, const uint64_t* starts, uint64_t m, int model,
                    orc_record* records, uint64_t* words, uint64_t cap_words) {
  if (m == 0) {
    uint64_t nw = orc_words_for_bits(0);
    if (cap_words < nw) return 0;
    memset(words, 0, nw * sizeof(uint64_t));
    return nw;
  }
  if (starts[0] != 0 || starts[m] != n) orc_die("bad partition bounds");
  if (model != ORC_MODEL_CONSTANT && model != ORC_MODEL_LINEAR && model != ORC_MODEL_POLY) orc_die("model");
  orc_choice* ch = (orc_choice*)malloc(sizeof(orc_choice) * m);
  if (!ch) orc_die("oom");
  uint64_t off = 0;
  for (uint64_t p = 0; p < m; p++) {
    uint64_t a = starts[p], e = starts[p + 1];
    if (e <= a) orc_die("empty partition");
    if (model == ORC_MODEL_POLY) {
      orc_choose_model(v + a, e - a, &ch[p]);
    } else {
      memset(&ch[p], 0, sizeof(ch[p]));
      ch[p].kind = model;
      orc_fit_partition(v + a, e - a, model, &ch[p].fit);
    }
    records[p].start = a;
    if (ch[p].kind >= 2) {
      records[p].theta0 = 0.0;
      records[p].theta1 = 0.0;
      records[p].word3 = make_word3(off, ch[p].poly.b, 0, 0) | ((uint64_t)1 << 63);
      off += 320 + (e - a) * (uint64_t)ch[p].poly.b;
    } else {
      records[p].theta0 = ch[p].fit.theta0;
      records[p].theta1 = ch[p].fit.theta1;
      records[p].word3 = make_word3(off, ch[p].fit.b, ch[p].fit.s, ch[p].fit.exact);
      off += (e - a) * (uint64_t)ch[p].fit.b;
    }
  }
  if (off >= ((uint64_t)1 << 48)) orc_die("stream longer than 2^48 bits");
  uint64_t nw = orc_words_for_bits(off);
  if (cap_words < nw) {
    free(ch);
    return 0;
  }
  memset(words, 0, nw * sizeof(uint64_t));
  for (uint64_t p = 0; p < m; p++) {
    uint64_t a = starts[p], e = starts[p + 1], N = e - a;
    uint64_t pos = records[p].word3 & (((uint64_t)1 << 48) - 1);
    int b;
    if (ch[p].kind >= 2) {
      const orc_poly_fit* q = &ch[p].poly;
      put_field(words, pos, 64, (uint64_t)q->T);
      for (int j = 1; j <= 3; j++) put_field(words, pos + 64 * (uint64_t)j, 64, (uint64_t)q->K[j]);
      put_field(words, pos + 256, 64, (uint64_t)q->sj[1] | ((uint64_t)q->sj[2] << 8) | ((uint64_t)q->sj[3] << 16));
      pos += 320;
      b = q->b;
    } else {
      b = ch[p].fit.b;
    }
    for (uint64_t x = 0; x < N; x++) {
      uint64_t pred;
      if (ch[p].kind >= 2)
        pred = (uint64_t)ch[p].poly.T + (uint64_t)poly_line(ch[p].poly.K, ch[p].poly.sj, ch[p].poly.S, N, x);
      else
        pred = (uint64_t)orc_predict(records[p].theta0, records[p].theta1, x);
      uint64_t z = zigzag64((int64_t)(v[a + x] - pred));
      if (b < 64 && (z >> b) != 0) orc_die("residual wider than b");
      put_field(words, pos + x * (uint64_t)b, b, z);
    }
  }
  free(ch);
  return nw;
}

/* ------------------------------------------------------------ decoder (§3.3) */

static int rec_b(const orc_record* r) { return (int)((r->word3 >> 48) & 0x7F); }
static uint64_t rec_off(const orc_record* r) { return r->word3 & (((uint64_t)1 << 48) - 1); }

static int rec_poly(const orc_record* r) { return (int)(r->word3 >> 63); }

/* Value at local index x of a partition of N values: prediction + unzigzag(bits [off + b x, +b)).
   A polynomial partition (R10) reads T, K1..K3 and the exponent word at off, its residuals from
   off + 320. */
static uint64_t decode_one(const orc_record* r, const uint64_t* words, uint64_t N, uint64_t x) {
  int b = rec_b(r);
  uint64_t pos = rec_off(r);
  uint64_t pred;
  if (rec_poly(r)) {
    int64_t K[4] = {0, 0, 0, 0};
    int32_t sj[4] = {0, 0, 0, 0}, S = 0;
    uint64_t T = get_field(words, pos, 64);
    uint64_t E = get_field(words, pos + 256, 64);
    for (int j = 1; j <= 3; j++) {
      K[j] = (int64_t)get_field(words, pos + 64 * (uint64_t)j, 64);
      sj[j] = (int32_t)((E >> (8 * (j - 1))) & 0xFF);
      if (sj[j] > S) S = sj[j];
    }
    pred = T + (uint64_t)poly_line(K, sj, S, N, x);
    pos += 320;
  } else {
    pred = (uint64_t)orc_predict(r->theta0, r->theta1, x);
  }
  uint64_t z = get_field(words, pos + x * (uint64_t)b, b);
  return pred + (uint64_t)unzigzag64(z);
}

/* Range decompression = the point decode applied to every position (§3.3). out: n values. */
void orc_decode(const orc_record* records, uint64_t m, const uint64_t* words, uint64_t n,
                int dtype_bits, uint64_t* out) {
  for (uint64_t p = 0; p < m; p++) {
    uint64_t a = records[p].start;
    uint64_t e = p + 1 < m ? records[p + 1].start : n;
    for (uint64_t i = a; i < e; i++) {
      uint64_t val = decode_one(&records[p], words, e - a, i - a);
      out[i] = dtype_bits == 32 ? (val & 0xFFFFFFFFu) : val;
    }
  }
}

/* partition holding position i: fixed -> i / L; variable -> largest start <= i (§3.3) */
static uint64_t find_partition(const orc_record* records, uint64_t m, uint32_t L, uint64_t i) {
  if (L > 0) return i / L;
  uint64_t lo = 0, hi = m; /* invariant: records[lo].start <= i < records[hi].start */
  while (hi - lo > 1) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (records[mid].start <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

/*
 * Point lookups (§3.3 Decoder). L > 0: fixed partitions of length L; L == 0: variable, searched
 * over the record starts. An index >= n yields 0 and counts as out of range. Returns the count of
 * out-of-range indices.
 */
uint64_t orc_lookup(const orc_record* records, uint64_t m, const uint64_t* words, uint64_t n,
                    uint32_t L, int dtype_bits, const uint64_t* idx, uint64_t k, uint64_t* out) {
  uint64_t bad = 0;
  for (uint64_t q = 0; q < k; q++) {
    uint64_t i = idx[q];
    if (i >= n) {
      out[q] = 0;
      bad++;
      continue;
    }
    uint64_t p = find_partition(records, m, L, i);
    uint64_t e = p + 1 < m ? records[p + 1].start : n;
    uint64_t val = decode_one(&records[p], words, e - records[p].start, i - records[p].start);
    out[q] = dtype_bits == 32 ? (val & 0xFFFFFFFFu) : val;
  }
  return bad;
}

/*
 * Filter + aggregate over the column: count and sum of the values v with lo <= v <= hi compared
 * as unsigned, sum exact mod 2^128 (the scan of §5.1 without pruning). out = {count, sum_lo, sum_hi}.
 */
void orc_filter_sum(const orc_record* records, uint64_t m, const uint64_t* words, uint64_t n,
                    int dtype_bits, uint64_t lo, uint64_t hi, uint64_t* out) {
  uint64_t count = 0;
  u128 sum = 0;
  for (uint64_t p = 0; p < m; p++) {
    uint64_t a = records[p].start;
    uint64_t e = p + 1 < m ? records[p + 1].start : n;
    for (uint64_t i = a; i < e; i++) {
      uint64_t val = decode_one(&records[p], words, e - a, i - a);
      if (dtype_bits == 32) val &= 0xFFFFFFFFu;
      if (val >= lo && val <= hi) {
        count++;
        sum += val;
      }
    }
  }
  out[0] = count;
  out[1] = (uint64_t)sum;
  out[2] = (uint64_t)(sum >> 64);
}

/* ------------------------------------------------------------ variable-length partitioner (§3.2.2) */

/* delta-tilde(v[i,j)) = bitlen(max d - min d) over d_k = w_k - w_{k-1}, i < k < j (R7) */
int orc_delta_tilde(const uint64_t* v, uint64_t i, uint64_t j) {
  if (j < i + 2) return 0;
  i128 mx = 0, mn = 0;
  for (uint64_t k = i + 1; k < j; k++) {
    i128 d = (i128)(int64_t)v[k] - (i128)(int64_t)v[k - 1];
    if (k == i + 1 || d > mx) mx = d;
    if (k == i + 1 || d < mn) mn = d;
  }
  return bitlen_u128((u128)(mx - mn));
}

/* Delta-encoding width of v[i,j): max bitlen(zigzag(d_k)) over i < k < j (§2, §3.2.2 example) */
int orc_delta_bits(const uint64_t* v, uint64_t i, uint64_t j) {
  int best = 0;
  for (uint64_t k = i + 1; k < j; k++) {
    int64_t d = (int64_t)(v[k] - v[k - 1]);
    int bl = bitlen_u64(zigzag64(d));
    if (bl > best) best = bl;
  }
  return best;
}

#define ORC_METRIC_TILDE 0 /* the linear regressor's fast metric */
#define ORC_METRIC_DELTA 1 /* Delta encoding's implicit step model */

static int metric_of(const uint64_t* v, uint64_t i, uint64_t j, int metric) {
  return metric == ORC_METRIC_DELTA ? orc_delta_bits(v, i, j) : orc_delta_tilde(v, i, j);
}

/* Space cost of adding v_j to the partition v[i,j): C = (j+1-i) D(v[i,j+1)) - (j-i) D(v[i,j)) */
int64_t orc_split_cost(const uint64_t* v, uint64_t i, uint64_t j, int metric) {
  return (int64_t)(j + 1 - i) * metric_of(v, i, j + 1, metric) -
         (int64_t)(j - i) * metric_of(v, i, j, metric);
}

/*
 * Split phase (§3.2.2, R7): one left-to-right sweep; v_j joins the open partition [i, j) iff
 * C <= tau * S_M and the partition is shorter than cap; otherwise v_j opens a new partition. A
 * chunk boundary (multiples of chunk; chunk = 0 means none) always opens a new partition.
 * starts_out receives m+1 entries (the last is n); returns m.
 */
uint64_t orc_var_split(const uint64_t* v, uint64_t n, double tau, uint64_t sm_bits, uint64_t cap,
                       uint64_t chunk, int metric, uint64_t* starts_out) {
  if (n == 0) {
    starts_out[0] = 0;
    return 0;
  }
  double thresh = tau * (double)sm_bits;
  uint64_t m = 0;
  uint64_t i = 0; /* open partition [i, j) */
  starts_out[m++] = 0;
  /* running max/min of the inner differences d_{i+1..j-1} of the open partition */
  i128 dmax = 0, dmin = 0;
  int cur = 0; /* metric of v[i, j) */
  for (uint64_t j = 1; j < n; j++) {
    int take = 1;
    if ((chunk && j % chunk == 0) || j - i >= cap) take = 0;
    int next = 0;
    i128 nmax = dmax, nmin = dmin;
    if (take) {
      if (metric == ORC_METRIC_DELTA) {
        int64_t d = (int64_t)(v[j] - v[j - 1]);
        int bl = bitlen_u64(zigzag64(d));
        next = bl > cur ? bl : cur;
      } else {
        i128 d = (i128)(int64_t)v[j] - (i128)(int64_t)v[j - 1];
        if (j == i + 1) {
          nmax = nmin = d;
        } else {
          if (d > nmax) nmax = d;
          if (d < nmin) nmin = d;
        }
        next = bitlen_u128((u128)(nmax - nmin));
      }
      int64_t C = (int64_t)(j + 1 - i) * next - (int64_t)(j - i) * cur;
      if (!((double)C <= thresh)) take = 0;
    }
    if (take) {
      cur = next;
      dmax = nmax;
      dmin = nmin;
    } else {
      starts_out[m++] = j;
      i = j;
      cur = 0;
      dmax = dmin = 0;
    }
  }
  starts_out[m] = n;
  return m;
}

/*
 * Seed of the chunk [a, e) for the seeded split (§3.2.2 "selecting good starting positions", R11):
 * the first k in [a, e-3] whose second-order delta w_{k+2} - 2 w_{k+1} + w_k needs the fewest bits
 * as a zigzag code (the linear regressor's smoothest window); a for chunks of fewer than 3 values.
 */
uint64_t orc_chunk_seed(const uint64_t* v, uint64_t a, uint64_t e) {
  if (e - a < 3) return a;
  uint64_t best = a;
  int best_bits = 1000;
  for (uint64_t k = a; k + 2 < e; k++) {
    i128 d2 = (i128)(int64_t)v[k + 2] - 2 * (i128)(int64_t)v[k + 1] + (i128)(int64_t)v[k];
    u128 z = d2 >= 0 ? (u128)d2 * 2 : (u128)(-d2) * 2 - 1;
    int bits = bitlen_u128(z);
    if (bits < best_bits) {
      best_bits = bits;
      best = k;
    }
  }
  return best;
}

/*
 * Seeded split (R11): per chunk, partitions grow away from the chunk's seed in both directions:
 * [seed, e) by the greedy sweep of orc_var_split, and [a, seed) by the same sweep run on its values
 * in reverse order (a partition that ends where the reversed sweep opened one starts right after
 * it). The chunk edge and the seed always start a partition. starts_out needs n+1 entries;
 * returns m.
 */
uint64_t orc_var_split_seeded(const uint64_t* v, uint64_t n, double tau, uint64_t sm_bits, uint64_t cap,
                              uint64_t chunk, int metric, uint64_t* starts_out) {
  if (n == 0) {
    starts_out[0] = 0;
    return 0;
  }
  if (chunk == 0) chunk = n;
  uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (chunk + 1));
  uint64_t* rev = (uint64_t*)malloc(sizeof(uint64_t) * (chunk + 1));
  if (!tmp || !rev) orc_die("oom");
  uint64_t m = 0;
  for (uint64_t a = 0; a < n; a += chunk) {
    uint64_t e = a + chunk < n ? a + chunk : n;
    uint64_t seed = orc_chunk_seed(v, a, e);
    if (seed > a) {
      uint64_t len = seed - a;
      for (uint64_t k = 0; k < len; k++) rev[k] = v[seed - 1 - k];
      uint64_t q = orc_var_split(rev, len, tau, sm_bits, cap, 0, metric, tmp);
      /* reversed partition [tmp[r], tmp[r+1]) = original [seed - tmp[r+1], seed - tmp[r]) */
      for (uint64_t r = q; r >= 1; r--) starts_out[m++] = seed - tmp[r];
    }
    uint64_t q = orc_var_split(v + seed, e - seed, tau, sm_bits, cap, 0, metric, tmp);
    for (uint64_t r = 0; r < q; r++) starts_out[m++] = seed + tmp[r];
  }
  starts_out[m] = n;
  free(tmp);
  free(rev);
  return m;
}

/* size in bits of v[a, e) with the full regressor: S_M + len * b (§3.2.2 merge) */
static uint64_t seg_size(const uint64_t* v, uint64_t a, uint64_t e, int model, uint64_t sm_bits) {
  orc_fit f;
  orc_fit_partition(v + a, e - a, model, &f);
  return sm_bits + (e - a) * (uint64_t)f.b;
}

/*
 * Merge phase, the paper's reading (R8 seq): scan left to right; merge the current partition with
 * its right neighbour when the merged size is smaller than the two apart, and then try the merged
 * one with its new neighbour; otherwise move on. Repeat whole passes until a pass merges nothing.
 * In place on starts (m+1 entries); returns the new m.
 */
uint64_t orc_var_merge_seq(const uint64_t* v, uint64_t* starts, uint64_t m, int model,
                           uint64_t sm_bits, uint64_t cap, uint64_t* passes_out) {
  uint64_t passes = 0;
  if (m < 2) {
    if (passes_out) *passes_out = 0;
    return m;
  }
  uint64_t* sz = (uint64_t*)malloc(sizeof(uint64_t) * m);
  if (!sz) orc_die("oom");
  for (uint64_t p = 0; p < m; p++) sz[p] = seg_size(v, starts[p], starts[p + 1], model, sm_bits);
  int changed = 1;
  while (changed) {
    changed = 0;
    passes++;
    /* the current partition is [starts[k], starts[j]) with size cur; kept partitions go to 0..k */
    uint64_t k = 0;
    uint64_t cur = sz[0];
    for (uint64_t j = 1; j < m; j++) {
      uint64_t a = starts[k], c = starts[j + 1];
      if (c - a <= cap) {
        uint64_t merged = seg_size(v, a, c, model, sm_bits);
        if (merged < cur + sz[j]) {
          cur = merged; /* partition j joins the current one */
          changed = 1;
          continue;
        }
      }
      sz[k] = cur;
      k++;
      starts[k] = starts[j];
      cur = sz[j];
    }
    sz[k] = cur;
    starts[k + 1] = starts[m];
    m = k + 1;
  }
  free(sz);
  if (passes_out) *passes_out = passes;
  return m;
}

/* SplitMix64 (Steele, Lea & Flood 2014): first output of the generator seeded with x. Used only
   as a fixed tie-break priority for equal merge gains. */
uint64_t orc_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* priority of pair j: gain first, then the hash of the pair's start position, then the position */
static int pair_beats(int64_t g1, uint64_t pos1, int64_t g2, uint64_t pos2) {
  if (g1 != g2) return g1 > g2;
  uint64_t h1 = orc_splitmix64(pos1), h2 = orc_splitmix64(pos2);
  if (h1 != h2) return h1 > h2;
  return pos1 < pos2;
}

/*
 * Merge phase, round-synchronous reading (R8 round): per round, gain g_j = size(P_j) +
 * size(P_{j+1}) - size(P_j u P_{j+1}) for every adjacent pair (pairs longer than cap have no
 * gain); every pair with g_j > 0 whose priority (g_j, splitmix64(start of P_j)) beats both
 * neighbouring pairs is merged at once (no two such pairs share a partition); stop when a round
 * selects nothing. Returns the new m; rounds_out gets the number of rounds that merged something.
 */
uint64_t orc_var_merge_round(const uint64_t* v, uint64_t* starts, uint64_t m, int model,
                             uint64_t sm_bits, uint64_t cap, uint64_t* rounds_out) {
  uint64_t rounds = 0;
  if (m < 2) {
    if (rounds_out) *rounds_out = 0;
    return m;
  }
  uint64_t* sz = (uint64_t*)malloc(sizeof(uint64_t) * m);
  uint64_t* msz = (uint64_t*)malloc(sizeof(uint64_t) * m);
  int64_t* gain = (int64_t*)malloc(sizeof(int64_t) * m);
  unsigned char* sel = (unsigned char*)malloc(m);
  uint64_t* nst = (uint64_t*)malloc(sizeof(uint64_t) * (m + 1));
  uint64_t* nsz = (uint64_t*)malloc(sizeof(uint64_t) * m);
  if (!sz || !msz || !gain || !sel || !nst || !nsz) orc_die("oom");
  for (uint64_t p = 0; p < m; p++) sz[p] = seg_size(v, starts[p], starts[p + 1], model, sm_bits);
  const int64_t NONE = INT64_MIN;
  for (;;) {
    for (uint64_t j = 0; j + 1 < m; j++) {
      uint64_t a = starts[j], c = starts[j + 2];
      if (c - a > cap) {
        gain[j] = NONE;
        continue;
      }
      msz[j] = seg_size(v, a, c, model, sm_bits);
      gain[j] = (int64_t)(sz[j] + sz[j + 1]) - (int64_t)msz[j];
    }
    uint64_t nsel = 0;
    for (uint64_t j = 0; j + 1 < m; j++) {
      int64_t g = gain[j];
      int ok = g != NONE && g > 0;
      if (ok && j > 0 && !pair_beats(g, starts[j], gain[j - 1], starts[j - 1])) ok = 0;
      if (ok && j + 2 < m && !pair_beats(g, starts[j], gain[j + 1], starts[j + 1])) ok = 0;
      sel[j] = (unsigned char)ok;
      nsel += (uint64_t)ok;
    }
    if (nsel == 0) break;
    rounds++;
    uint64_t k = 0;
    for (uint64_t j = 0; j < m; j++) {
      nst[k] = starts[j];
      if (j + 1 < m && sel[j]) {
        nsz[k] = msz[j];
        j++; /* partition j+1 joins j */
      } else {
        nsz[k] = sz[j];
      }
      k++;
    }
    nst[k] = starts[m];
    m = k;
    memcpy(starts, nst, sizeof(uint64_t) * (m + 1));
    memcpy(sz, nsz, sizeof(uint64_t) * m);
    if (m < 2) break;
  }
  free(sz);
  free(msz);
  free(gain);
  free(sel);
  free(nst);
  free(nsz);
  if (rounds_out) *rounds_out = rounds;
  return m;
}

/* ------------------------------------------------------------ partition-size search (§3.2.1) */

/*
 * Sample of the column for the fixed-partition size search (§3.2.1, step 1): subsequences of
 * length N (the largest partition size searched) whose starts are SplitMix64(seed + i) mod
 * (n - N + 1) for i = 0 .. k-1, with k = max(1, floor(frac * n / N)), so at most a fraction frac of
 * the values (plus one subsequence) is sampled. A column of at most N values is its own only
 * sample (N is then n). Writes the k starts; returns k.
 */
uint64_t orc_search_samples(uint64_t n, uint64_t N, double frac, uint64_t seed, uint64_t* starts_out) {
  if (n <= N) {
    starts_out[0] = 0;
    return 1;
  }
  uint64_t k = (uint64_t)(frac * (double)n / (double)N);
  if (k < 1) k = 1;
  for (uint64_t i = 0; i < k; i++) starts_out[i] = orc_splitmix64(seed + i) % (n - N + 1);
  return k;
}

/* Compressed size (bits) of the samples under fixed partitions of size L: each subsequence is cut
 * into partitions of L values from its own start (the last may be short), each costing
 * S_M + len * b (§3, the size function). */
uint64_t orc_sample_size_bits(const uint64_t* v, const uint64_t* starts, uint64_t k, uint64_t N, uint64_t L,
                              int model) {
  uint64_t total = 0;
  for (uint64_t s = 0; s < k; s++)
    for (uint64_t a = 0; a < N; a += L) {
      const uint64_t len = a + L <= N ? L : N - a;
      total += orc_partition_size_bits(v + starts[s] + a, len, model);
    }
  return total;
}

/*
 * The search (§3.2.1, steps 2-3), in this reading:
 *  - exponential phase: L = 1, 2, 4, ... (powers of two up to N, then N itself), stopping after the
 *    first size above its predecessor's: the sizes are U-shaped in L, so that step is past the
 *    minimum;
 *  - back search: from the best L so far, probe L - step and L + step (inside [1, N]) with step
 *    starting at half the best L; move to the smaller size when it is smaller, else halve the step;
 *  - stop when the step reaches 0, or when a move improves the size by less than 0.01 %
 *    (old - new < old / 10^4, in integers).
 * Sizes are cached per L. Returns the chosen L; *best_bits gets its sample size and *evals the
 * number of distinct L evaluated.
 */
uint64_t orc_search_partition_size(const uint64_t* v, uint64_t n, uint64_t N, double frac, uint64_t seed,
                                   int model, uint64_t* best_bits, uint64_t* evals) {
  if (n == 0) {
    if (best_bits) *best_bits = 0;
    if (evals) *evals = 0;
    return 1;
  }
  if (n < N) N = n;
  uint64_t kmax = (uint64_t)(frac * (double)n / (double)N);
  if (kmax < 1) kmax = 1;
  uint64_t* starts = (uint64_t*)malloc(sizeof(uint64_t) * kmax);
  uint64_t* cache = (uint64_t*)calloc(N + 1, sizeof(uint64_t)); /* 0 = not evaluated */
  if (!starts || !cache) orc_die("out of memory");
  const uint64_t k = orc_search_samples(n, N, frac, seed, starts);
  uint64_t ne = 0;
#define SIZE_AT(LL) (cache[LL] ? cache[LL] : (ne++, cache[LL] = orc_sample_size_bits(v, starts, k, N, LL, model) + 1))
  /* cache holds size + 1 so that 0 marks "not evaluated" */
  uint64_t best = 1, best_s = SIZE_AT(1);
  uint64_t prev_s = best_s;
  for (uint64_t L = 2;; L *= 2) {
    const uint64_t LL = L < N ? L : N;
    const uint64_t s = SIZE_AT(LL);
    if (s < best_s) {
      best_s = s;
      best = LL;
    }
    if (s > prev_s || LL == N) break;
    prev_s = s;
  }
  for (uint64_t step = best / 2; step > 0;) {
    uint64_t cand = best, cand_s = best_s;
    if (best > step) {
      const uint64_t s = SIZE_AT(best - step);
      if (s < cand_s) {
        cand_s = s;
        cand = best - step;
      }
    }
    if (best + step <= N) {
      const uint64_t s = SIZE_AT(best + step);
      if (s < cand_s) {
        cand_s = s;
        cand = best + step;
      }
    }
    if (cand == best) {
      step /= 2;
      continue;
    }
    const int small_gain = (best_s - cand_s) * 10000 < best_s - 1; /* cached sizes are size + 1 */
    best = cand;
    best_s = cand_s;
    if (small_gain) break;
  }
#undef SIZE_AT
  free(starts);
  free(cache);
  if (best_bits) *best_bits = best_s - 1;
  if (evals) *evals = ne;
  return best;
}
