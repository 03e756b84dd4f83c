// Tiled column scans (§3.3 range decompression; the filter + sum of §5.1 without materialising
// values): full/range decode and the fused filter-sum.
//
// Tile t covers positions [t kScanTile, (t+1) kScanTile); its residuals are one contiguous bit
// range. A persistent CTA has one producer warp and four or eight consumer warps. The producer
// walks the CTA's tiles in order: it waits until a shared-memory stage is empty, then issues one
// 1-D bulk copy (TMA) of the tile's 16-byte-aligned word range and one of its decode-table entries
// (when at most kMaxP partitions touch it), completing on the stage's "full" mbarrier; tiles that
// pruning removes never enter the ring. Each consumer warp decodes 4096 / (consumer warps)
// positions of the tile lane-strided (lane j takes positions g + j), so global stores
// are coalesced and neighbouring fields are read from shared memory without bank conflicts. Inside
// a partition a lane carries its fixed-point prediction F = A + B x and its bit position, stepping
// by 32 B and 32 b per group. The filter bounds each 32-value group with its model (prediction at
// both ends +- the residual range of width b) and decodes only groups that can meet [lo, hi].
// Tile descriptors (word range, partitions, value bounds) are built once per column.
#include <string.h>

#include "leco_internal.cuh"
#include "tma.cuh"

namespace leco {

namespace {

constexpr int kMaxStages = 8;
constexpr int kMaxConsumerWarps = 8;
constexpr int kMaxP = 64;
constexpr uint32_t kAuxBytes = kMaxP * 32;

enum Mode { kDecode64 = 0, kDecode32 = 1, kFilter = 2, kDecodeAny = 3 };

struct TileMeta {
  uint64_t p0;
  uint64_t bit_base;  // absolute bit position of the first staged word
  uint32_t np;
  uint32_t staged;    // decode-table entries p0 .. p0+np-1 are in shared memory
  uint32_t skip;      // pruned: the job is dropped, nothing is copied
  uint32_t cls;       // filter: 1 = the tile misses [lo, hi], 2 = lies inside it, 0 = undecided
  uint32_t end;       // no job: the producer has no more work for this CTA
};

struct ScanArgs {
  ColumnView c;
  uint64_t begin, end;       // positions to emit
  uint64_t t_first, t_last;  // tiles touching [begin, end)
  void* out;                 // decode output: position i -> out[i - begin]
  uint64_t lo, hi;           // filter range
  uint32_t flags;
  leco_sum_result* res;
};

// what a consumer needs for one staged tile (written by the producer into the stage's slot)
struct Job {
  TileMeta mt;
  ScanArgs g;
  uint64_t tile;
};

struct Ctrl {
  uint64_t full[kMaxStages];
  uint64_t empty[kMaxStages];
  uint64_t red[3][kMaxConsumerWarps];
  uint64_t issued;
  uint64_t consumed[kMaxConsumerWarps];
  int abort;
  Job job[kMaxStages];
};

constexpr uint32_t kCtrlBytes = (sizeof(Ctrl) + 127) & ~127u;

__device__ __forceinline__ uint64_t pstart(const ColumnView& c, uint64_t p) {
  if (c.starts) return __ldg(c.starts + p);
  const uint64_t s = p * (uint64_t)c.L;
  return s < c.n ? s : c.n;
}

// partition holding position i, searched inside [lo, hi) (hi exclusive, i >= start(lo))
__device__ __forceinline__ uint64_t part_of(const ColumnView& c, uint64_t i, uint64_t lo, uint64_t hi) {
  if (!c.starts) return c.n <= 0xFFFFFFFFull ? (uint64_t)((uint32_t)i / c.L) : i / c.L;
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(c.starts + mid) <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ Aux ldg_aux(const Aux* a) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(a);
  const ulonglong2 v0 = __ldg(q), v1 = __ldg(q + 1);
  Aux r;
  r.A = (int64_t)v0.x;
  r.B = (int64_t)v0.y;
  r.start = v1.x;
  r.word3 = v1.y;
  return r;
}

// Model bounds of positions [x0, x1] of an exact partition: the value w = pred + r satisfies
// pmin - 2^(b-1) <= w <= pmax + 2^(b-1) - 1 as a signed integer, with the prediction taken at both
// ends (it is monotone in x) and r in the zigzag range of width b. Returned as a set of unsigned
// values: kind 1 = [vlo, vhi]; kind 2 = [0, vhi] together with [vlo, 2^64 - 1] (a 64-bit range that
// straddles zero as a signed number); kind 0 = no bound (binary64 partition, b > 62, or an
// extreme range). A 32-bit column's values are w itself, in [0, 2^32), so its range is clamped.
__device__ __forceinline__ int part_bounds(int dtype, const Aux& a, uint64_t x0, uint64_t x1,
                                           uint64_t* vlo_out, uint64_t* vhi_out) {
  const uint32_t b = w3_b(a.word3);
  if (!w3_exact(a.word3) || b > 62) return 0;
  int32_t sh = w3_s(a.word3);
  sh = (sh > 0 ? sh : 0) & 63;
  const int64_t p0v = (int64_t)((uint64_t)a.A + (uint64_t)a.B * x0) >> sh;
  const int64_t p1v = (int64_t)((uint64_t)a.A + (uint64_t)a.B * x1) >> sh;
  const int64_t pmin = p0v < p1v ? p0v : p1v, pmax = p0v < p1v ? p1v : p0v;
  const int64_t half = b ? (int64_t)1 << (b - 1) : 0;
  if (pmin < INT64_MIN + half || pmax > INT64_MAX - half) return 0;
  const int64_t L = pmin - half, U = pmax + (half ? half - 1 : 0);
  if (dtype == LECO_U32) {
    const int64_t lo = L > 0 ? L : 0, hi = U < 0xFFFFFFFFll ? U : 0xFFFFFFFFll;
    if (lo > hi) return 0;
    *vlo_out = (uint64_t)lo;
    *vhi_out = (uint64_t)hi;
    return 1;
  }
  *vlo_out = (uint64_t)L;
  *vhi_out = (uint64_t)U;
  return (L < 0 && U >= 0) ? 2 : 1;
}

// Union of a tile's running bound set (kind k, [lo, hi]) with one partition's (kind pk, [plo, phi]).
__device__ __forceinline__ int bounds_union(int k, uint64_t* lo, uint64_t* hi, int pk, uint64_t plo, uint64_t phi) {
  if (k == 0 || pk == 0) return 0;
  if (k == 1 && pk == 1) {
    *lo = min(*lo, plo);
    *hi = max(*hi, phi);
    return 1;
  }
  if (k == 1) {  // make the running set the wrapped one
    const uint64_t t0 = *lo, t1 = *hi;
    *lo = plo;
    *hi = phi;
    plo = t0;
    phi = t1;
    pk = 1;
  }
  if (pk == 2) {
    *hi = max(*hi, phi);
    *lo = min(*lo, plo);
  } else if (plo < *lo) {  // [plo, phi] lies in [0, max(hi, phi)] (plo >= 0)
    *hi = max(*hi, phi);
  }
  return *hi < *lo - 1 ? 2 : 0;  // the two pieces met: no bound left
}

// 0 = may meet [lo, hi], 1 = certainly misses, 2 = certainly inside
__device__ __forceinline__ int classify(int kind, uint64_t vlo, uint64_t vhi, uint64_t lo, uint64_t hi) {
  if (kind == 1) {
    if (vhi < lo || vlo > hi) return 1;
    if (vlo >= lo && vhi <= hi) return 2;
    return 0;
  }
  if (kind == 2 && lo > vhi && hi < vlo) return 1;
  return 0;
}

// b-bit field (b <= 32) at bit position bit of a staged word buffer
__device__ __forceinline__ uint32_t field32(const uint32_t* w, uint32_t bit, uint32_t mask) {
  const uint32_t k = bit >> 5;
  return __funnelshift_r(w[k], w[k + 1], bit) & mask;
}

// b-bit field (32 < b <= 64)
__device__ __forceinline__ uint64_t field64(const uint32_t* w, uint32_t bit, uint64_t mask) {
  const uint32_t k = bit >> 5;
  const uint32_t w0 = w[k], w1 = w[k + 1], w2 = w[k + 2];
  const uint32_t lo = __funnelshift_r(w0, w1, bit);
  const uint32_t hi = __funnelshift_r(w1, w2, bit);
  return (((uint64_t)hi << 32) | lo) & mask;
}

__device__ __forceinline__ int64_t unzigzag32(uint32_t z) {
  return (int64_t)(int32_t)((z >> 1) ^ (0u - (z & 1u)));
}

// the same residual mod 2^32
__device__ __forceinline__ uint32_t unzigzag_u32(uint32_t z) { return (z >> 1) ^ (0u - (z & 1u)); }

struct Acc {
  uint64_t cnt = 0, lo = 0, hi = 0;
  __device__ __forceinline__ void add(uint64_t v) {
    cnt++;
    const uint64_t t = lo + v;
    hi += t < lo ? 1ull : 0ull;
    lo = t;
  }
};

template <int MODE>
__device__ __forceinline__ void emit(const ScanArgs& g, Acc& acc, uint64_t i, uint64_t v, uint64_t vmask) {
  if (MODE == kDecode64) {
    reinterpret_cast<uint64_t*>(g.out)[i - g.begin] = v;
  } else if (MODE == kDecode32) {
    reinterpret_cast<uint32_t*>(g.out)[i - g.begin] = (uint32_t)v;
  } else {
    v &= vmask;
    if (v >= g.lo && v <= g.hi) acc.add(v);
  }
}

// one position decoded from scratch (partition search, multiply): boundary groups only. ANY_MODEL:
// the column may hold polynomial partitions (single-column scans of constant and linear columns
// leave that branch out)
template <bool ANY_MODEL>
__device__ __forceinline__ uint64_t value_at(const ScanArgs& g, const uint32_t* words, const Aux* saux,
                                             const TileMeta& mt, uint64_t i, uint64_t q) {
  const ColumnView& c = g.c;
  Aux a;
  if (mt.staged) {
    const uint64_t last = mt.p0 + mt.np - 1;
    while (q < last && saux[q + 1 - mt.p0].start <= i) q++;
    a = saux[q - mt.p0];
  } else {
    q = part_of(c, i, q, mt.p0 + mt.np);
    a = ldg_aux(c.aux + q);
  }
  const uint64_t x = i - a.start;
  const uint32_t b = w3_b(a.word3);
  const uint32_t bit = (uint32_t)(w3_off(a.word3) + (uint64_t)b * x - mt.bit_base);
  const uint64_t z = b <= 32 ? (uint64_t)field32(words, bit, (uint32_t)low_mask(b)) : field64(words, bit, low_mask(b));
  const int64_t pred = ANY_MODEL ? predict_aux(a, c.rec, c.poly, q, x) : predict_aux_line(a, c.rec, q, x);
  return (uint64_t)pred + (uint64_t)zz_decode(z);
}

// Tight loop over ng whole 32-value groups of one exact partition (the common case), then a
// partial group whose first `tail` lanes hold the partition's (or the warp range's) last values.
// Lane j handles positions i0 + j + 32 k; its fixed-point prediction F and bit position step by
// 32 B and 32 b. Filter runs are classified once by their model bounds: missed runs cost nothing,
// runs certainly inside are summed without the compare.
template <int MODE, bool WIDE, bool ZERO_B>
__device__ __forceinline__ void run_groups(const ScanArgs& g, Acc& acc, const uint32_t* words,
                                           const Aux& a, uint64_t i0, uint32_t ng, uint32_t tail,
                                           uint64_t bit_base, uint32_t lane, int cls) {
  const uint32_t b = w3_b(a.word3);
  int32_t sh = w3_s(a.word3);
  sh = (sh > 0 ? sh : 0) & 63;
  const uint64_t x = i0 + lane - a.start;
  uint64_t F = (uint64_t)a.A + (uint64_t)a.B * x;
  const uint64_t B32 = (uint64_t)a.B * 32u;
  uint32_t bit = (uint32_t)(w3_off(a.word3) + (uint64_t)b * x - bit_base);
  const uint32_t b32 = 32u * b;
  const uint64_t mask64 = low_mask(b);
  const uint32_t mask32 = (uint32_t)mask64;
  if (ZERO_B && (MODE == kDecode64 || MODE == kDecode32) && b == 0) {
    // every residual is zero: the values are the predictions (columns with short partitions, where
    // such runs are common)
    const uint32_t steps = ng + (lane < tail ? 1u : 0u);
    if (MODE == kDecode64) {
      uint64_t* o = reinterpret_cast<uint64_t*>(g.out) + (i0 + lane - g.begin);
      for (uint32_t k = 0; k < steps; k++, o += 32, F += B32) *o = (uint64_t)((int64_t)F >> sh);
    } else {
      uint32_t* o = reinterpret_cast<uint32_t*>(g.out) + (i0 + lane - g.begin);
      for (uint32_t k = 0; k < steps; k++, o += 32, F += B32) *o = (uint32_t)(uint64_t)((int64_t)F >> sh);
    }
    return;
  }
  if (MODE == kDecode64) {
    uint64_t* o = reinterpret_cast<uint64_t*>(g.out) + (i0 + lane - g.begin);
#pragma unroll 4
    for (uint32_t k = 0; k < ng; k++) {
      const int64_t r = WIDE ? zz_decode(field64(words, bit, mask64)) : unzigzag32(field32(words, bit, mask32));
      *o = (uint64_t)(((int64_t)F >> sh) + r);
      o += 32;
      F += B32;
      bit += b32;
    }
    if (lane < tail) {
      const int64_t r = WIDE ? zz_decode(field64(words, bit, mask64)) : unzigzag32(field32(words, bit, mask32));
      *o = (uint64_t)(((int64_t)F >> sh) + r);
    }
  } else if (MODE == kDecode32) {
    uint32_t* o = reinterpret_cast<uint32_t*>(g.out) + (i0 + lane - g.begin);
#pragma unroll 4
    for (uint32_t k = 0; k < ng; k++) {
      const uint32_t r = WIDE ? (uint32_t)zz_decode(field64(words, bit, mask64)) : unzigzag_u32(field32(words, bit, mask32));
      *o = (uint32_t)(uint64_t)((int64_t)F >> sh) + r;  // floor: arithmetic shift
      o += 32;
      F += B32;
      bit += b32;
    }
    if (lane < tail) {
      const uint32_t r = WIDE ? (uint32_t)zz_decode(field64(words, bit, mask64)) : unzigzag_u32(field32(words, bit, mask32));
      *o = (uint32_t)(uint64_t)((int64_t)F >> sh) + r;
    }
  } else {
    const uint64_t vmask = g.c.dtype == LECO_U32 ? 0xFFFFFFFFull : ~0ull;
    if (cls == 1) return;
    const uint32_t steps = ng + (lane < tail ? 1u : 0u);
    if (cls == 2) {
      for (uint32_t k = 0; k < steps; k++) {
        const int64_t r = WIDE ? zz_decode(field64(words, bit, mask64)) : unzigzag32(field32(words, bit, mask32));
        acc.add((uint64_t)(((int64_t)F >> sh) + r) & vmask);
        F += B32;
        bit += b32;
      }
      return;
    }
    for (uint32_t k = 0; k < steps; k++) {
      const int64_t r = WIDE ? zz_decode(field64(words, bit, mask64)) : unzigzag32(field32(words, bit, mask32));
      const uint64_t v = (uint64_t)(((int64_t)F >> sh) + r) & vmask;
      if (v >= g.lo && v <= g.hi) acc.add(v);
      F += B32;
      bit += b32;
    }
  }
}

// Tight loop over ng whole 32-value groups of one polynomial partition (§3.1 polynomial terms):
// lane j's prediction T + (F(x) >> S) steps by forward differences of the cubic F over strides of
// 32 positions, exactly in 128-bit two's complement arithmetic (the differences start from F at
// x, x + 32, x + 64, x + 96 by Horner's rule). F and its differences are carried multiplied by
// 2^(64-S) modulo 2^128: floor(F / 2^S) mod 2^64 is then the high half of the carried value, so
// the loop shifts nothing. Filter runs have no model bounds: every value is compared.
template <int MODE, bool WIDE>
__device__ __forceinline__ void run_groups_poly(const ScanArgs& g, Acc& acc, const uint32_t* words,
                                                const Aux& a, uint64_t q, uint64_t i0, uint32_t ng,
                                                uint64_t bit_base, uint32_t lane) {
  const uint32_t b = w3_b(a.word3);
  const int32_t S = w3_s(a.word3) & 63;
  const uint64_t x = i0 + lane - a.start;
  const ulonglong2* row = reinterpret_cast<const ulonglong2*>(g.c.poly + q);
  u128 c[4];
  for (int k = 0; k < 4; k++) {
    const ulonglong2 h = __ldg(row + k);
    c[k] = ((u128)h.y << 64) | h.x;
  }
  // F(x) and its forward differences over the stride h = 32, in closed form:
  // D1 = a1 h + a2 (2xh + h^2) + a3 (3x^2 h + 3x h^2 + h^3), D2 = a2 2h^2 + a3 (6x h^2 + 6h^3),
  // D3 = a3 6h^3 (x < 2^14, so every bracket fits 64 bits)
  const uint64_t h = 32;
  const uint32_t up = 64u - (uint32_t)S;  // 2..64
  u128 F = (((c[3] * x + c[2]) * x + c[1]) * x + c[0]) << up;
  u128 D1 = (c[1] * h + c[2] * (2 * x * h + h * h) + c[3] * (3 * x * x * h + 3 * x * h * h + h * h * h)) << up;
  u128 D2 = (c[2] * (2 * h * h) + c[3] * (6 * x * h * h + 6 * h * h * h)) << up;
  const u128 D3 = (c[3] * (6 * h * h * h)) << up;
  uint32_t bit = (uint32_t)(w3_off(a.word3) + (uint64_t)b * x - bit_base);
  const uint32_t b32 = 32u * b;
  const uint64_t mask64 = low_mask(b);
  const uint32_t mask32 = (uint32_t)mask64;
  const uint64_t T = (uint64_t)a.A;
  if (MODE == kDecode64 || MODE == kDecode32) {
    const uint64_t o0 = i0 + lane - g.begin;
    for (uint32_t k = 0; k < ng; k++) {
      const int64_t r = WIDE ? zz_decode(field64(words, bit, mask64)) : unzigzag32(field32(words, bit, mask32));
      const uint64_t v = T + (uint64_t)(F >> 64) + (uint64_t)r;
      if (MODE == kDecode64)
        reinterpret_cast<uint64_t*>(g.out)[o0 + 32ull * k] = v;
      else
        reinterpret_cast<uint32_t*>(g.out)[o0 + 32ull * k] = (uint32_t)v;
      F += D1;
      D1 += D2;
      D2 += D3;
      bit += b32;
    }
  } else {
    const uint64_t vmask = g.c.dtype == LECO_U32 ? 0xFFFFFFFFull : ~0ull;
    for (uint32_t k = 0; k < ng; k++) {
      const int64_t r = WIDE ? zz_decode(field64(words, bit, mask64)) : unzigzag32(field32(words, bit, mask32));
      const uint64_t v = (T + (uint64_t)(F >> 64) + (uint64_t)r) & vmask;
      if (v >= g.lo && v <= g.hi) acc.add(v);
      F += D1;
      D1 += D2;
      D2 += D3;
      bit += b32;
    }
  }
}

// TAIL: an exact run goes to its end, its last group partial, and the next run starts at the
// partition's edge (columns whose partition edges fall anywhere); otherwise a run stops at its last
// whole group and a group across an edge is decoded position by position (fixed partitions of a
// multiple of 32 values, whose edges meet the warp ranges' 32-value grid).
template <int MODE, bool POLY, bool TAIL>
__device__ void process_tile(const ScanArgs& g, uint64_t t, const TileMeta& mt, const uint32_t* words,
                             const Aux* saux, Acc& acc, uint32_t per_warp) {
  const ColumnView& c = g.c;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint64_t tile_base = t * kScanTile;
  const uint64_t wbeg = max(g.begin, tile_base + (uint64_t)warp * per_warp);
  const uint64_t wend = min(min(g.end, c.n), tile_base + (uint64_t)(warp + 1) * per_warp);
  const uint64_t vmask = c.dtype == LECO_U32 ? 0xFFFFFFFFull : ~0ull;
  const uint64_t last = mt.p0 + mt.np - 1;
  uint64_t q = mt.p0;
  uint64_t gp = wbeg;
  while (gp < wend) {
    // partition holding gp (warp-uniform)
    Aux a;
    if (mt.staged) {
      while (q < last && saux[q + 1 - mt.p0].start <= gp) q++;
      a = saux[q - mt.p0];
    } else {
      q = part_of(c, gp, q, mt.p0 + mt.np);
      a = ldg_aux(c.aux + q);
    }
    const uint64_t qend = (q < last && mt.staged) ? saux[q + 1 - mt.p0].start : pstart(c, q + 1);
    const uint64_t run_end = min(qend, wend);
    const uint32_t ng = (uint32_t)((run_end - gp) >> 5);
    if (ng && w3_exact(a.word3)) {
      const uint32_t tail = TAIL ? (uint32_t)(run_end - gp) & 31u : 0u;
      const uint64_t last_x = (TAIL ? run_end : gp + 32ull * ng) - 1 - a.start;
      int cls = (int)mt.cls;
      if (MODE == kFilter && cls == 0 && !(g.flags & LECO_FILTER_DECODE_ALL)) {
        uint64_t vlo = 0, vhi = 0;
        const int kind = part_bounds(c.dtype, a, gp - a.start, last_x, &vlo, &vhi);
        cls = classify(kind, vlo, vhi, g.lo, g.hi);
      }
      if (w3_b(a.word3) > 32)
        run_groups<MODE, true, false>(g, acc, words, a, gp, ng, tail, mt.bit_base, lane, cls);
      else
        run_groups<MODE, false, TAIL>(g, acc, words, a, gp, ng, tail, mt.bit_base, lane, cls);
      gp = TAIL ? run_end : gp + 32ull * ng;
    } else if (POLY && ng && w3_poly(a.word3)) {
      if (w3_b(a.word3) > 32)
        run_groups_poly<MODE, true>(g, acc, words, a, q, gp, ng, mt.bit_base, lane);
      else
        run_groups_poly<MODE, false>(g, acc, words, a, q, gp, ng, mt.bit_base, lane);
      gp += 32ull * ng;
    } else {
      // a group that crosses a partition end, a partial last group, a binary64 partition, or a
      // polynomial partition in a kernel without the polynomial loop: each lane decodes its
      // position from scratch
      const uint64_t i = gp + lane;
      if (i < wend) emit<MODE>(g, acc, i, value_at<POLY>(g, words, saux, mt, i, q), vmask);
      gp += 32;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Producer side for one job: the staged tile's metadata from its descriptor, plus the filter
// classification (and pruning) for this range.
__device__ __forceinline__ TileMeta meta_from(const TileDesc& d, int mode, const ScanArgs& g) {
  TileMeta mt;
  mt.p0 = d.p0;
  mt.np = d.np;
  mt.staged = d.np <= (uint32_t)kMaxP;
  mt.bit_base = d.g0 * 8;
  mt.cls = 0;
  if (mode == kFilter && !(g.flags & LECO_FILTER_DECODE_ALL))
    mt.cls = (uint32_t)classify((int)d.bounds, d.vmin, d.vmax, g.lo, g.hi);
  mt.skip = ((g.flags & LECO_FILTER_PRUNE) && mt.cls == 1) ? 1u : 0u;
  mt.end = 0;
  return mt;
}

// Persistent scan. One producer warp (the last) and CW consumer warps; nst stages of stage_bytes
// word bytes + the decode-table slot. MULTI: jobs come from a work table (column, tile, range,
// output) over several columns; otherwise every tile of [g.begin, g.end) of the one column g.c.
// POLY: the column (or a column of the batch) may hold polynomial partitions, decoded by their own
// loop (a separate instantiation, so that constant and linear columns keep the smaller register
// budget).
template <int MODE, int CW, bool MULTI, bool POLY, bool TAIL>
__global__ void __launch_bounds__((CW + 1) * 32)
    k_tilescan(const ScanArgs g0, const ColumnView* __restrict__ cols, const BatchItem* __restrict__ items,
               uint64_t nitems, uint32_t nst, uint32_t stage_bytes) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Ctrl& ctl = *reinterpret_cast<Ctrl*>(smem_raw);
  const uint32_t stride = stage_bytes + kAuxBytes;
  unsigned char* stages = smem_raw + kCtrlBytes;
  const uint64_t njobs = MULTI ? nitems : g0.t_last - g0.t_first + 1;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < nst; s++) {
      mbar_init(&ctl.full[s], 1);
      mbar_init(&ctl.empty[s], CW);
    }
    ctl.abort = 0;
    ctl.issued = 0;
    mbar_fence_init();
  }
  if (threadIdx.x < CW) ctl.consumed[threadIdx.x] = 0;
  __syncthreads();

  if (warp == CW) {
    // producer: the warp's lanes fetch 32 jobs' descriptors at a time and classify them in
    // parallel; a pruned job is dropped here and never occupies a stage. In turn, lane j (which
    // holds job j's descriptor in registers) waits for its stage to drain and issues the job's
    // copies, so no global load sits between consecutive copies. A final job marked `end` tells
    // the consumers to stop.
    uint64_t it = 0;
    uint32_t s = 0, ph = 0;  // stage of copy `it` and the parity of its round (it / nst)
    bool stop = false;
    for (uint64_t k0 = blockIdx.x; k0 < njobs && !stop; k0 += 32ull * gridDim.x) {
      const uint64_t kk = k0 + (uint64_t)lane * gridDim.x;
      ScanArgs mine = g0;
      uint64_t tile = 0;
      TileDesc d = {};
      TileMeta mt = {};
      if (kk < njobs) {
        if (MULTI) {
          const BatchItem bi = items[kk];
          mine.c = cols[bi.col];
          mine.begin = bi.begin;
          mine.end = bi.end;
          mine.out = bi.out;
          tile = bi.tile;
        } else {
          tile = g0.t_first + kk;
        }
        d = mine.c.tiles[tile];
        mt = meta_from(d, MODE, mine);
      }
      uint32_t todo = __ballot_sync(0xffffffffu, kk < njobs && !mt.skip);
      while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1;
        int ok = 1;
        if (lane == (uint32_t)j) {
          if (it >= (uint64_t)nst) ok = mbar_wait_bounded(&ctl.empty[s], ph ^ 1u) ? 1 : 0;
          if (ok && *(volatile int*)&ctl.abort) ok = 0;
          if (!ok) {
            atomicOr(g0.c.status, kStatTimeout);
            *(volatile int*)&ctl.abort = 1;
          } else {
            // publish the job into the drained slot, then arm the stage and issue its copies
            Job& jb = ctl.job[s];
            if (MULTI) jb.g = mine;  // a single-column scan's consumers take the arguments from g0
            jb.tile = tile;
            jb.mt = mt;
            unsigned char* dst = stages + (size_t)s * stride;
            const uint32_t abytes = mt.staged ? mt.np * 32u : 0u;
            mbar_arrive_expect_tx(&ctl.full[s], d.wbytes + abytes);
            bulk_g2s(dst, reinterpret_cast<const char*>(mine.c.words) + d.g0, d.wbytes, &ctl.full[s]);
            if (abytes) bulk_g2s(dst + stage_bytes, mine.c.aux + mt.p0, abytes, &ctl.full[s]);
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, j);
        if (!ok) {
          stop = true;
          break;
        }
        it++;
        if (++s == nst) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    if (lane == 0) {
      ctl.issued = it;  // copies issued (each one's stage is armed)
      bool ok = !stop;
      if (ok && it >= (uint64_t)nst) ok = mbar_wait_bounded(&ctl.empty[s], ph ^ 1u);
      if (ok) {
        ctl.job[s].mt.end = 1u;
        mbar_arrive(&ctl.full[s]);
      } else if (!stop) {
        atomicOr(g0.c.status, kStatTimeout);
        *(volatile int*)&ctl.abort = 1;
      }
    }
  } else {
    Acc acc;
    uint64_t it = 0;
    uint32_t s = 0, ph = 0;
    const uint32_t per_warp = (uint32_t)(kScanTile / CW);
    for (;;) {
      const bool ok = mbar_wait_bounded(&ctl.full[s], ph);
      if (!ok || *(volatile int*)&ctl.abort) {
        if (lane == 0) {
          atomicOr(g0.c.status, kStatTimeout);
          *(volatile int*)&ctl.abort = 1;
        }
        break;
      }
      const TileMeta mt = ctl.job[s].mt;
      if (mt.end) break;
      if (!(MODE == kFilter && mt.cls == 1)) {
        const ScanArgs g = MULTI ? ctl.job[s].g : g0;
        const uint64_t tile = ctl.job[s].tile;
        const unsigned char* base = stages + (size_t)s * stride;
        const uint32_t* words = reinterpret_cast<const uint32_t*>(base);
        const Aux* saux = reinterpret_cast<const Aux*>(base + stage_bytes);
        if (MODE == kDecodeAny) {
          if (g.c.dtype == LECO_U32)
            process_tile<kDecode32, POLY, TAIL>(g, tile, mt, words, saux, acc, per_warp);
          else
            process_tile<kDecode64, POLY, TAIL>(g, tile, mt, words, saux, acc, per_warp);
        } else {
          process_tile<MODE, POLY, TAIL>(g, tile, mt, words, saux, acc, per_warp);
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&ctl.empty[s]);
        ctl.consumed[warp] = it + 1;
      }
      it++;
      if (++s == nst) {
        s = 0;
        ph ^= 1u;
      }
    }
    if (MODE == kFilter) {
      uint64_t cnt = warp_sum_u64(acc.cnt);
      uint64_t lo = acc.lo, hi = acc.hi;
      for (int o = 16; o > 0; o >>= 1) {
        const uint64_t l2 = __shfl_down_sync(0xffffffffu, lo, o);
        const uint64_t h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const uint64_t nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
      }
      if (lane == 0) {
        ctl.red[0][warp] = cnt;
        ctl.red[1][warp] = lo;
        ctl.red[2][warp] = hi;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ctl.abort) {
      // a wait gave up: drain (bounded) the copies this CTA issued but nobody consumed
      uint64_t done = ctl.issued;
      for (int w = 0; w < CW; w++) done = min(done, ctl.consumed[w]);
      for (uint64_t u = done; u < ctl.issued; u++)
        mbar_wait_bounded(&ctl.full[u % nst], (uint32_t)((u / nst) & 1), 100000000ull);
    } else if (MODE == kFilter) {
      uint64_t tc = 0, tl = 0, th = 0;
      for (int w = 0; w < CW; w++) {
        tc += ctl.red[0][w];
        const uint64_t nl = tl + ctl.red[1][w];
        th += ctl.red[2][w] + (nl < tl ? 1ull : 0ull);
        tl = nl;
      }
      if (tc) {
        atomicAdd((unsigned long long*)&g0.res->count, (unsigned long long)tc);
        const unsigned long long old = atomicAdd((unsigned long long*)&g0.res->sum_lo, (unsigned long long)tl);
        const uint64_t carry = (old + tl < old) ? 1ull : 0ull;
        if (th + carry) atomicAdd((unsigned long long*)&g0.res->sum_hi, (unsigned long long)(th + carry));
      }
    }
  }
}

// one descriptor per tile: partitions, 16-byte-aligned word range, model value bounds
__device__ TileDesc tile_desc_one(const ColumnView& c, uint64_t t) {
  {
    const uint64_t i0 = t * kScanTile, i1 = min(i0 + kScanTile, c.n);
    const uint64_t p0 = part_of(c, i0, 0, c.m);
    const uint64_t p1 = part_of(c, i1 - 1, p0, c.m);
    const Aux a0 = ldg_aux(c.aux + p0);
    const Aux a1 = ldg_aux(c.aux + p1);
    const uint64_t bstart = w3_off(a0.word3) + (uint64_t)w3_b(a0.word3) * (i0 - a0.start);
    const uint64_t bend = w3_off(a1.word3) + (uint64_t)w3_b(a1.word3) * (i1 - a1.start);
    const uint64_t g0 = (bstart >> 7) << 4;
    const uint64_t g1 = ((bend + 64 + 127) >> 7) << 4;  // one extra 64-bit word for funnel reads
    TileDesc d;
    d.p0 = p0;
    d.np = (uint32_t)(p1 - p0 + 1);
    d.g0 = g0;
    d.wbytes = (uint32_t)(g1 - g0);
    d.pad = 0;
    uint64_t vmin = 0, vmax = 0;
    int kind = 0;
    for (uint64_t p = p0; p <= p1; p++) {
      const Aux a = p == p0 ? a0 : (p == p1 ? a1 : ldg_aux(c.aux + p));
      const uint64_t ps = max(i0, a.start);
      const uint64_t pe = min(i1, pstart(c, p + 1));
      uint64_t lo = 0, hi = 0;
      const int pk = part_bounds(c.dtype, a, ps - a.start, pe - 1 - a.start, &lo, &hi);
      if (p == p0) {
        kind = pk;
        vmin = lo;
        vmax = hi;
      } else {
        kind = bounds_union(kind, &vmin, &vmax, pk, lo, hi);
      }
      if (kind == 0) break;
    }
    d.bounds = (uint32_t)kind;
    d.vmin = kind ? vmin : 0;
    d.vmax = kind ? vmax : ~0ull;
    return d;
  }
}

__device__ __forceinline__ i128 shfl_down_i128(i128 v, int o) {
  const uint64_t lo = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)(u128)v, o);
  const uint64_t hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)((u128)v >> 64), o);
  return (i128)(((u128)hi << 64) | lo);
}

__device__ __forceinline__ i128 shfl_lane0_i128(i128 v) {
  const uint64_t lo = __shfl_sync(0xffffffffu, (unsigned long long)(uint64_t)(u128)v, 0);
  const uint64_t hi = __shfl_sync(0xffffffffu, (unsigned long long)(uint64_t)((u128)v >> 64), 0);
  return (i128)(((u128)hi << 64) | lo);
}

// Bounds of the values at local positions [xa, xb) of polynomial partition p (warp-collective; the
// result in every lane): each lane enumerates floor(F(x) / 2^S) for x = xa + lane + 32k by forward
// differences of F, the warp takes the exact min and max, and the residual range of width b widens
// them: T + min - 2^(b-1) <= w <= T + max + 2^(b-1) - 1. Kinds as part_bounds.
__device__ int poly_part_bounds(const ColumnView& c, const Aux& a, uint64_t p, uint64_t xa, uint64_t xb,
                                uint32_t lane, uint64_t* vlo_out, uint64_t* vhi_out) {
  const uint32_t b = w3_b(a.word3);
  const int32_t S = w3_s(a.word3) & 63;
  const ulonglong2* row = reinterpret_cast<const ulonglong2*>(c.poly + p);
  u128 cf[4];
  for (int k = 0; k < 4; k++) {
    const ulonglong2 h = __ldg(row + k);
    cf[k] = ((u128)h.y << 64) | h.x;
  }
  const uint64_t x = xa + lane, h = 32;
  u128 F = ((cf[3] * x + cf[2]) * x + cf[1]) * x + cf[0];
  u128 D1 = cf[1] * h + cf[2] * (2 * x * h + h * h) + cf[3] * (3 * x * x * h + 3 * x * h * h + h * h * h);
  u128 D2 = cf[2] * (2 * h * h) + cf[3] * (6 * x * h * h + 6 * h * h * h);
  const u128 D3 = cf[3] * (6 * h * h * h);
  i128 qmin = ((i128)1 << 126), qmax = -((i128)1 << 126);
  for (uint64_t xx = x; xx < xb; xx += 32) {
    const i128 q = (i128)F >> S;
    qmin = q < qmin ? q : qmin;
    qmax = q > qmax ? q : qmax;
    F += D1;
    D1 += D2;
    D2 += D3;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const i128 m0 = shfl_down_i128(qmin, o), m1 = shfl_down_i128(qmax, o);
    qmin = m0 < qmin ? m0 : qmin;
    qmax = m1 > qmax ? m1 : qmax;
  }
  qmin = shfl_lane0_i128(qmin);
  qmax = shfl_lane0_i128(qmax);
  if (b > 62 || xa >= xb) return 0;
  const i128 half = b ? (i128)1 << (b - 1) : 0;
  const i128 L = (i128)a.A + qmin - half, U = (i128)a.A + qmax + (half ? half - 1 : 0);
  if (L < (i128)INT64_MIN || U > (i128)INT64_MAX) return 0;
  if (c.dtype == LECO_U32) {
    const i128 lo = L > 0 ? L : 0, hi = U < (i128)0xFFFFFFFFll ? U : (i128)0xFFFFFFFFll;
    if (lo > hi) return 0;
    *vlo_out = (uint64_t)lo;
    *vhi_out = (uint64_t)hi;
    return 1;
  }
  *vlo_out = (uint64_t)(int64_t)L;
  *vhi_out = (uint64_t)(int64_t)U;
  return (L < 0 && U >= 0) ? 2 : 1;
}

// Value bounds of the tiles of a column with polynomial partitions (a warp per tile): the bounds
// k_tile_desc leaves out for polynomial partitions (their predictions are not monotone), from the
// exact predictions; partitions with a line keep part_bounds. Tiles without a polynomial partition
// are left as they are.
__device__ void tile_poly_bounds_one(const ColumnView& c, TileDesc* __restrict__ tiles, uint64_t t, uint32_t lane) {
  const uint64_t p0 = tiles[t].p0, np = tiles[t].np;
  bool any = false;
  for (uint64_t p = p0; p < p0 + np && !any; p++) any = w3_poly(ldg_aux(c.aux + p).word3) != 0;
  if (!any) return;
  const uint64_t i0 = t * kScanTile, i1 = min(i0 + kScanTile, c.n);
  int kind = 0;
  uint64_t vmin = 0, vmax = 0;
  for (uint64_t p = p0; p < p0 + np; p++) {
    const Aux a = ldg_aux(c.aux + p);
    const uint64_t ps = max(i0, a.start), pe = min(i1, pstart(c, p + 1));
    uint64_t lo = 0, hi = 0;
    const int pk = w3_poly(a.word3) ? poly_part_bounds(c, a, p, ps - a.start, pe - a.start, lane, &lo, &hi)
                                    : part_bounds(c.dtype, a, ps - a.start, pe - 1 - a.start, &lo, &hi);
    if (p == p0) {
      kind = pk;
      vmin = lo;
      vmax = hi;
    } else {
      kind = bounds_union(kind, &vmin, &vmax, pk, lo, hi);
    }
    if (kind == 0) break;
  }
  if (lane == 0) {
    tiles[t].bounds = (uint32_t)kind;
    tiles[t].vmin = kind ? vmin : 0;
    tiles[t].vmax = kind ? vmax : ~0ull;
  }
}

__global__ void k_tile_poly_bounds(const ColumnView c, TileDesc* __restrict__ tiles) {
  const uint64_t nt = scan_tiles(c.n);
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t t = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < nt; t += nw)
    tile_poly_bounds_one(c, tiles, t, threadIdx.x & 31u);
}

// the same over the tiles of a batch of columns (columns without a polynomial table are skipped)
__global__ void k_tile_poly_bounds_multi(const ColumnView* __restrict__ views, const uint64_t* __restrict__ tile_base,
                                         uint32_t ncols, uint64_t T, TileDesc* __restrict__ tiles) {
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t g = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g < T; g += nw) {
    const uint32_t c = find_col(tile_base, ncols, g);
    const ColumnView v = views[c];
    if (v.poly) tile_poly_bounds_one(v, tiles + tile_base[c], g - tile_base[c], threadIdx.x & 31u);
  }
}

__global__ void k_tile_desc(const ColumnView c, TileDesc* __restrict__ tiles) {
  const uint64_t nt = scan_tiles(c.n);
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nt;
       t += (uint64_t)gridDim.x * blockDim.x)
    tiles[t] = tile_desc_one(c, t);
}

__global__ void k_tile_desc_multi(const ColumnView* __restrict__ views, const uint64_t* __restrict__ tile_base,
                                  uint32_t ncols, uint64_t T, TileDesc* __restrict__ tiles) {
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < T;
       g += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = find_col(tile_base, ncols, g);
    tiles[g] = tile_desc_one(views[c], g - tile_base[c]);
  }
}

template <int MODE, int CW, bool MULTI, bool POLY, bool TAIL>
cudaError_t launch_scan_cfg(const ScanArgs& g, const ColumnView* cols, const BatchItem* items,
                            uint64_t nitems, uint32_t stage_bytes, ScanConfig cfg, cudaStream_t st) {
  const uint32_t nst = cfg.stages < 2 ? 2u : (cfg.stages > (uint32_t)kMaxStages ? (uint32_t)kMaxStages : cfg.stages);
  const uint32_t smem = kCtrlBytes + nst * (stage_bytes + kAuxBytes);
  auto kern = k_tilescan<MODE, CW, MULTI, POLY, TAIL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, (CW + 1) * 32, smem);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  const uint64_t njobs = MULTI ? nitems : g.t_last - g.t_first + 1;
  const uint64_t cap = (uint64_t)sm_count() * nb;
  const unsigned grid = (unsigned)(njobs < cap ? njobs : cap);
  kern<<<grid, (CW + 1) * 32, smem, st>>>(g, cols, items, nitems, nst, stage_bytes);
  return cudaGetLastError();
}

// poly: the column (a single-column scan: it has a polynomial table) or some column of the batch
// may hold polynomial partitions
// (a multi-column scan, and a column with polynomial partitions, always end runs at partition edges)
template <int MODE, bool MULTI>
cudaError_t launch_scan(const ScanArgs& g, const ColumnView* cols, const BatchItem* items, uint64_t nitems,
                        uint32_t stage_bytes, ScanConfig cfg, bool poly, cudaStream_t st) {
  if (poly) {
    if (cfg.consumer_warps == 4)
      return launch_scan_cfg<MODE, 4, MULTI, true, true>(g, cols, items, nitems, stage_bytes, cfg, st);
    return launch_scan_cfg<MODE, 8, MULTI, true, true>(g, cols, items, nitems, stage_bytes, cfg, st);
  }
  const bool grid32 = !MULTI && !g.c.starts && g.c.L % 32 == 0;  // every partition edge on the 32-value grid
  if (grid32) {
    if (cfg.consumer_warps == 4)
      return launch_scan_cfg<MODE, 4, MULTI, false, false>(g, cols, items, nitems, stage_bytes, cfg, st);
    return launch_scan_cfg<MODE, 8, MULTI, false, false>(g, cols, items, nitems, stage_bytes, cfg, st);
  }
  if (cfg.consumer_warps == 4)
    return launch_scan_cfg<MODE, 4, MULTI, false, true>(g, cols, items, nitems, stage_bytes, cfg, st);
  return launch_scan_cfg<MODE, 8, MULTI, false, true>(g, cols, items, nitems, stage_bytes, cfg, st);
}

// One CTA waits on an mbarrier that nothing arrives at: the bounded wait must give up after limit_ns
// and record kStatTimeout, the same path a scan takes when a copy never lands.
__global__ void k_wait_selftest(uint64_t limit_ns, uint32_t* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, kStatTimeout);
}

}  // namespace

cudaError_t launch_wait_selftest(uint64_t limit_ns, uint32_t* status, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, status);
  return cudaGetLastError();
}

cudaError_t launch_tile_desc(const ColumnView& c, TileDesc* tiles, cudaStream_t st) {
  const uint64_t nt = scan_tiles(c.n);
  if (nt == 0) return cudaSuccess;
  const uint64_t want = (nt + 127) / 128, cap = (uint64_t)sm_count() * 8;
  k_tile_desc<<<(int)(want < cap ? want : cap), 128, 0, st>>>(c, tiles);
  if (c.poly) {
    const uint64_t wb = (nt + 7) / 8;
    k_tile_poly_bounds<<<(int)(wb < cap ? wb : cap), 256, 0, st>>>(c, tiles);
  }
  return cudaGetLastError();
}

cudaError_t launch_tile_desc_multi(const ColumnView* views, const uint64_t* tile_base, uint32_t ncols, uint64_t T,
                                   bool poly, TileDesc* tiles, cudaStream_t st) {
  if (T == 0) return cudaSuccess;
  const uint64_t want = (T + 127) / 128, cap = (uint64_t)sm_count() * 8;
  k_tile_desc_multi<<<(int)(want < cap ? want : cap), 128, 0, st>>>(views, tile_base, ncols, T, tiles);
  if (poly) {
    const uint64_t wb = (T + 7) / 8;
    k_tile_poly_bounds_multi<<<(int)(wb < cap ? wb : cap), 256, 0, st>>>(views, tile_base, ncols, T, tiles);
  }
  return cudaGetLastError();
}

cudaError_t launch_decode(const ColumnView& c, uint64_t begin, uint64_t count, void* out,
                          cudaStream_t st) {
  return launch_decode_cfg(c, begin, count, out, scan_config_for(c, 0), st);
}

cudaError_t launch_decode_cfg(const ColumnView& c, uint64_t begin, uint64_t count, void* out,
                              ScanConfig cfg, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  ScanArgs g;
  g.c = c;
  g.begin = begin;
  g.end = begin + count;
  g.t_first = begin / kScanTile;
  g.t_last = (begin + count - 1) / kScanTile;
  g.out = out;
  g.lo = g.hi = 0;
  g.flags = 0;
  g.res = nullptr;
  const bool poly = c.poly != nullptr;
  return c.dtype == LECO_U32 ? launch_scan<kDecode32, false>(g, nullptr, nullptr, 0, c.stage_bytes, cfg, poly, st)
                             : launch_scan<kDecode64, false>(g, nullptr, nullptr, 0, c.stage_bytes, cfg, poly, st);
}

cudaError_t launch_filter_sum(const ColumnView& c, uint64_t lo, uint64_t hi, uint32_t flags,
                              leco_sum_result* out, cudaStream_t st) {
  return launch_filter_sum_cfg(c, lo, hi, flags, out, scan_config_for(c, 1), st);
}

cudaError_t launch_filter_sum_cfg(const ColumnView& c, uint64_t lo, uint64_t hi, uint32_t flags,
                                  leco_sum_result* out, ScanConfig cfg, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(leco_sum_result), st);
  if (e != cudaSuccess || c.n == 0 || lo > hi) return e;
  ScanArgs g;
  g.c = c;
  g.begin = 0;
  g.end = c.n;
  g.t_first = 0;
  g.t_last = (c.n - 1) / kScanTile;
  g.out = nullptr;
  g.lo = lo;
  g.hi = hi;
  g.flags = flags;
  g.res = out;
  return launch_scan<kFilter, false>(g, nullptr, nullptr, 0, c.stage_bytes, cfg, c.poly != nullptr, st);
}

cudaError_t launch_batch_decode(const ColumnView* d_cols, const BatchItem* d_items, uint64_t nitems,
                                uint32_t stage_bytes, ScanConfig cfg, bool poly, uint32_t* status, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  ScanArgs g;
  memset(&g, 0, sizeof(g));
  g.c.status = status;
  return launch_scan<kDecodeAny, true>(g, d_cols, d_items, nitems, stage_bytes, cfg, poly, st);
}

}  // namespace leco
