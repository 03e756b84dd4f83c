// Encoder kernels (§3.1 Regressor, §3.3 Encoder): per-partition fit (fit.cuh), offset scan,
// decode-table build and residual packing.
#include "fit.cuh"
#include "leco_internal.cuh"
#include "tma.cuh"

namespace leco {

namespace {

constexpr int kFitBlock = 256;
constexpr int kFitWarps = kFitBlock / 32;
// CTAs of kFitBlock threads per SM for the fit (registers capped to fit them): the fit is bound by
// instruction issue, so more resident warps beat keeping every partition in flight inside L2
constexpr int kFitCtasPerSm = 4;

__device__ __forceinline__ uint64_t part_begin(const uint64_t* starts, uint32_t L, uint64_t n,
                                               uint64_t p) {
  if (starts) return starts[p];
  const uint64_t s = p * (uint64_t)L;
  return s < n ? s : n;
}

// ------------------------------------------------------------------------------ staged partitions
//
// The fit and the packing read each partition's values twice or more, so a CTA stages the
// partition in shared memory first: one 1-D bulk copy (TMA) of the 16-byte-aligned byte range
// around it, completing on an mbarrier, double-buffered so the copy of the CTA's next partition
// runs while the current one is processed. A partition the copy cannot take (the aligned range
// would leave the array, or it does not fit a buffer) is read with plain loads: into the buffer
// when it fits, else straight from global memory by the body.

constexpr uint32_t kStageData = 32768;             // partition bytes one buffer holds
constexpr uint32_t kStageBuf = kStageData + 32;    // + alignment lead and tail

// the value at position x of a partition staged in shared memory (raw values of the column's type)
__device__ __forceinline__ int64_t staged_value(const unsigned char* stage, int dtype, uint32_t x) {
  return dtype == LECO_U32 ? (int64_t)reinterpret_cast<const uint32_t*>(stage)[x]
                           : reinterpret_cast<const int64_t*>(stage)[x];
}

struct PartSrc {
  const void* values;  // the column's values
  uint64_t n;          // values in the column
  uint64_t a;          // first position of the partition
  uint32_t N;          // its length
  int dtype;
};

// aligned byte range [g0, g0 + bytes) of the column holding the partition (at most cap value bytes);
// lead = the partition's offset inside it
__device__ __forceinline__ bool stage_plan(const PartSrc& s, uint32_t cap, uint64_t* g0, uint32_t* bytes,
                                           uint32_t* lead) {
  const uint64_t vb = s.dtype == LECO_U32 ? 4 : 8;
  if (s.N == 0 || (uint64_t)s.N * vb > cap || (reinterpret_cast<uintptr_t>(s.values) & 15u)) return false;
  const uint64_t b0 = s.a * vb, b1 = (s.a + s.N) * vb;
  const uint64_t a0 = b0 & ~15ull, a1 = (b1 + 15) & ~15ull;
  if (a1 > s.n * vb) return false;
  *g0 = a0;
  *bytes = (uint32_t)(a1 - a0);
  *lead = (uint32_t)(b0 - a0);
  return true;
}

// every thread decides (identically) whether the copy is used; thread 0 issues it
__device__ __forceinline__ bool stage_issue(const PartSrc& s, uint32_t cap, unsigned char* dst, uint64_t* full) {
  uint64_t g0;
  uint32_t bytes, lead;
  if (!stage_plan(s, cap, &g0, &bytes, &lead)) return false;
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(full, bytes);
    bulk_g2s(dst, static_cast<const char*>(s.values) + g0, bytes, full);
  }
  return true;
}

// Runs body(p, src, stage) for partitions p = blockIdx.x, + gridDim.x, ... < P, where stage is the
// partition's values in shared memory (raw, the column's type; partitions of at most cap bytes,
// cap <= kStageData) or nullptr. NBUF = 2 copies the
// CTA's next partition while the current one is processed; NBUF = 1 keeps the CTA small (more CTAs
// per SM hide each other's copies instead). body must end with a __syncthreads(). On a copy that
// never lands the CTA records kStatTimeout in *err and stops.
template <int NBUF, typename GetPart, typename Body>
__device__ void for_each_staged(uint64_t P, uint32_t cap, GetPart get, Body body, unsigned char* ring, uint64_t* full,
                                uint32_t* err) {
  if (threadIdx.x == 0) {
    for (int k = 0; k < NBUF; k++) mbar_init(&full[k], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t ph = 0, armed = 0;  // bit k: buffer k's mbarrier parity / a copy into buffer k is pending
  uint32_t buf = 0;
  uint64_t p = blockIdx.x;
  if (p < P && stage_issue(get(p), cap, ring, &full[0])) armed = 1u;
  for (; p < P; p += gridDim.x, buf = NBUF == 2 ? buf ^ 1u : 0u) {
    // the buffer written next was released by the previous body's closing barrier
    const uint32_t nb = NBUF == 2 ? buf ^ 1u : 0u;
    const uint64_t pn = p + gridDim.x;
    if (NBUF == 2) {
      armed &= ~(1u << nb);
      if (pn < P && stage_issue(get(pn), cap, ring + nb * kStageBuf, &full[nb])) armed |= 1u << nb;
    }
    const PartSrc s = get(p);
    unsigned char* b = ring + buf * kStageBuf;
    const unsigned char* st = nullptr;
    if ((armed >> buf) & 1u) {
      const bool ok = mbar_wait_bounded(&full[buf], (ph >> buf) & 1u);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0 && err) atomicOr(err, kStatTimeout);
        if (NBUF == 2 && ((armed >> nb) & 1u)) mbar_wait_bounded(&full[nb], (ph >> nb) & 1u);
        return;
      }
      ph ^= 1u << buf;
      uint64_t g0;
      uint32_t bytes, lead;
      stage_plan(s, cap, &g0, &bytes, &lead);
      st = b + lead;
    } else if ((uint64_t)s.N * (s.dtype == LECO_U32 ? 4 : 8) <= cap) {
      if (s.dtype == LECO_U32) {
        uint32_t* d = reinterpret_cast<uint32_t*>(b);
        for (uint32_t x = threadIdx.x; x < s.N; x += blockDim.x)
          d[x] = __ldg(static_cast<const uint32_t*>(s.values) + s.a + x);
      } else {
        uint64_t* d = reinterpret_cast<uint64_t*>(b);
        for (uint32_t x = threadIdx.x; x < s.N; x += blockDim.x)
          d[x] = __ldg(static_cast<const uint64_t*>(s.values) + s.a + x);
      }
      __syncthreads();
      st = b;
    }
    body(p, s, st);
    if (NBUF == 1) {  // the single buffer is free again: start the CTA's next partition
      armed = 0;
      if (pn < P && stage_issue(get(pn), cap, ring, &full[0])) armed = 1u;
    }
  }
}

// One warp per partition (grid-stride over warps): the fit's reductions are warp shuffles and its
// parameter solve runs on one lane, so a warp waiting on its solve stalls only itself while the
// SM's other warps stream their partitions; the second pass re-reads the partition from L2.
__global__ void __launch_bounds__(kFitBlock, kFitCtasPerSm)
    k_fit(const void* __restrict__ values, int dtype, uint64_t n, const uint64_t* __restrict__ starts,
          uint32_t L, uint64_t m, int model, Record* __restrict__ rec, uint64_t* __restrict__ lenbits,
          uint32_t* __restrict__ max_b) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nw = (uint64_t)gridDim.x * kFitWarps;
  for (uint64_t p = (uint64_t)blockIdx.x * kFitWarps + (threadIdx.x >> 5); p < m; p += nw) {
    const uint64_t a = part_begin(starts, L, n, p);
    const uint32_t N = (uint32_t)(part_begin(starts, L, n, p + 1) - a);
    const FitResult R = fit_range<32>(values, dtype, a, N, model, lane, nullptr);
    if (lane == 0) {
      Record r;
      r.theta0 = R.theta0;
      r.theta1 = R.theta1;
      r.start = a;
      r.word3 = make_w3(0, R.b, R.s, 1);
      rec[p] = r;
      lenbits[p] = (uint64_t)N * R.b;
      if (R.b) atomicMax(max_b, R.b);
    }
  }
}

// Two warps per partition (four partitions per 256-thread CTA, each pair of warps synchronised by its
// own named barrier): as many warps stream as with one warp per partition, but half as many
// partitions are in flight, so the second pass finds the partition in L2 instead of DRAM.
constexpr int kFitPairs = kFitBlock / 64;

__global__ void __launch_bounds__(kFitBlock, kFitCtasPerSm)
    k_fit_pairs(const void* __restrict__ values, int dtype, uint64_t n, const uint64_t* __restrict__ starts,
                uint32_t L, uint64_t m, int model, Record* __restrict__ rec, uint64_t* __restrict__ lenbits,
                uint32_t* __restrict__ max_b) {
  __shared__ FitShared sm[kFitPairs];
  const uint32_t g = threadIdx.x >> 6, rank = threadIdx.x & 63u;
  const uint64_t ng = (uint64_t)gridDim.x * kFitPairs;
  for (uint64_t p = (uint64_t)blockIdx.x * kFitPairs + g; p < m; p += ng) {
    const uint64_t a = part_begin(starts, L, n, p);
    const uint32_t N = (uint32_t)(part_begin(starts, L, n, p + 1) - a);
    const FitResult R = fit_range<64>(values, dtype, a, N, model, rank, &sm[g], 1 + (int)g);
    if (rank == 0) {
      Record r;
      r.theta0 = R.theta0;
      r.theta1 = R.theta1;
      r.start = a;
      r.word3 = make_w3(0, R.b, R.s, 1);
      rec[p] = r;
      lenbits[p] = (uint64_t)N * R.b;
      if (R.b) atomicMax(max_b, R.b);
    }
  }
}

// The polynomial model (fit.cuh): four phases over all partitions, each its own kernel. Phases 1
// and 3 read the values (a warp per partition), phases 2 and 4 are a thread per partition. A map
// says where partition p's values are: one column (OneColumn), or the polynomial columns of a
// batch (BatchColumns; partitions of the batch's other columns are skipped).
struct OneColumn {
  const void* values;
  uint64_t n;
  const uint64_t* starts;
  uint32_t L;
  __device__ __forceinline__ bool get(uint64_t p, const void** v, uint64_t* a, uint32_t* N, uint32_t* slot) const {
    *v = values;
    *a = part_begin(starts, L, n, p);
    *N = (uint32_t)(part_begin(starts, L, n, p + 1) - *a);
    *slot = 0;
    return true;
  }
};

struct BatchColumns {
  const EncCol* cols;
  const uint64_t* part_base;
  uint32_t ncols;
  __device__ __forceinline__ bool get(uint64_t p, const void** v, uint64_t* a, uint32_t* N, uint32_t* slot) const {
    const uint32_t c = find_col(part_base, ncols, p);
    const EncCol col = cols[c];
    if (col.model != LECO_MODEL_POLY) return false;
    const uint64_t s = (p - part_base[c]) * (uint64_t)col.L;
    *v = col.values;
    *a = s;
    *N = (uint32_t)((s + col.L < col.n ? s + col.L : col.n) - s);
    *slot = c;
    return true;
  }
};

template <typename Map>
__global__ void __launch_bounds__(kFitBlock)
    k_poly_moments(const Map map, int dtype, uint64_t m, PolyMom* __restrict__ mom) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nw = (uint64_t)gridDim.x * kFitWarps;
  for (uint64_t p = (uint64_t)blockIdx.x * kFitWarps + (threadIdx.x >> 5); p < m; p += nw) {
    const void* v;
    uint64_t a;
    uint32_t N, slot;
    if (!map.get(p, &v, &a, &N, &slot)) continue;
    const PolyMom M = poly_moments_warp(v, dtype, a, N, lane);
    if (lane == 0) mom[p] = M;
  }
}

template <typename Map>
__global__ void k_poly_plan(const Map map, uint64_t m, const PolyMom* __restrict__ mom, PolyPlan* __restrict__ plan) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    const void* v;
    uint64_t a;
    uint32_t N, slot;
    if (map.get(p, &v, &a, &N, &slot)) plan[p] = poly_plan(mom[p], N);
  }
}

template <typename Map>
__global__ void __launch_bounds__(kFitBlock)
    k_poly_ranges(const Map map, int dtype, uint64_t m, const PolyPlan* __restrict__ plan, PolyRange* __restrict__ rng) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nw = (uint64_t)gridDim.x * kFitWarps;
  for (uint64_t p = (uint64_t)blockIdx.x * kFitWarps + (threadIdx.x >> 5); p < m; p += nw) {
    const void* v;
    uint64_t a;
    uint32_t N, slot;
    if (!map.get(p, &v, &a, &N, &slot)) continue;
    const PolyRange R = poly_ranges_warp(v, dtype, a, N, lane, plan + p);
    if (lane == 0) rng[p] = R;
  }
}

// the record (offset 0, set by the offset scan), stream bits, block and widest width of the choice
// (max_b[slot]: the column's)
template <typename Map>
__global__ void k_poly_choose(const Map map, uint64_t m, const PolyMom* __restrict__ mom,
                              const PolyPlan* __restrict__ plan, const PolyRange* __restrict__ rng,
                              Record* __restrict__ rec, uint64_t* __restrict__ lenbits, PolyCoef* __restrict__ pcoef,
                              uint32_t* __restrict__ max_b) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    const void* v;
    uint64_t a;
    uint32_t N, slot;
    if (!map.get(p, &v, &a, &N, &slot)) continue;
    const FitChoice C = poly_choose(mom[p], plan[p], rng[p], N);
    Record r;
    r.start = a;
    if (C.kind >= 2) {
      r.theta0 = 0.0;
      r.theta1 = 0.0;
      r.word3 = make_w3(0, C.b, 0, 0) | kPolyFlag;
      pcoef[p] = C.pc;
      lenbits[p] = kPolyBlockBits + (uint64_t)N * C.b;
    } else {
      r.theta0 = C.R.theta0;
      r.theta1 = C.R.theta1;
      r.word3 = make_w3(0, C.R.b, C.R.s, 1);
      lenbits[p] = (uint64_t)N * C.R.b;
    }
    rec[p] = r;
    if (C.b) atomicMax(max_b + slot, C.b);
  }
}

// ------------------------------------------------------------------------------ exclusive scan

constexpr int kPrefixBlock = 256;
constexpr int kPrefixItems = 8;
constexpr uint64_t kPrefixTile = kPrefixBlock * kPrefixItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* warp_tot,
                                                         uint64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    uint64_t t = lane < (kPrefixBlock / 32) ? warp_tot[lane] : 0;
    uint64_t ti = t;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    if (lane < (kPrefixBlock / 32)) warp_tot[lane] = ti - t;
    if (lane == (kPrefixBlock / 32) - 1) *total = ti;
  }
  __syncthreads();
  const uint64_t r = warp_tot[wid] + inc - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kPrefixBlock)
    k_prefix_tiles(const uint64_t* __restrict__ in, uint64_t count, uint64_t* __restrict__ tile_sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kPrefixTile;
  uint64_t s = 0;
  for (int k = 0; k < kPrefixItems; k++) {
    const uint64_t i = base + (uint64_t)k * kPrefixBlock + threadIdx.x;
    if (i < count) s += in[i];
  }
  s = warp_sum_u64(s);
  __shared__ uint64_t ws[kPrefixBlock / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int k = 0; k < kPrefixBlock / 32; k++) t += ws[k];
    tile_sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kPrefixBlock)
    k_prefix_top(uint64_t* __restrict__ tile_sums, uint64_t ntiles, uint64_t* __restrict__ total) {
  __shared__ uint64_t wt[kPrefixBlock / 32];
  __shared__ uint64_t tot;
  uint64_t carry = 0;
  for (uint64_t base = 0; base < ntiles; base += kPrefixBlock) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t v = i < ntiles ? tile_sums[i] : 0;
    const uint64_t ex = block_exclusive_scan(v, wt, &tot);
    if (i < ntiles) tile_sums[i] = carry + ex;
    __syncthreads();
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kPrefixBlock)
    k_prefix_apply(const uint64_t* __restrict__ in, uint64_t count,
                 const uint64_t* __restrict__ tile_prefix, uint64_t* __restrict__ out) {
  __shared__ uint64_t wt[kPrefixBlock / 32];
  __shared__ uint64_t tot;
  const uint64_t base = (uint64_t)blockIdx.x * kPrefixTile + (uint64_t)threadIdx.x * kPrefixItems;
  uint64_t v[kPrefixItems];
  uint64_t s = 0;
  for (int k = 0; k < kPrefixItems; k++) {
    const uint64_t i = base + k;
    v[k] = i < count ? in[i] : 0;
    s += v[k];
  }
  uint64_t run = block_exclusive_scan(s, wt, &tot) + tile_prefix[blockIdx.x];
  for (int k = 0; k < kPrefixItems; k++) {
    const uint64_t i = base + k;
    if (i < count) out[i] = run;
    run += v[k];
  }
}

__global__ void k_set_offsets(Record* __restrict__ rec, const uint64_t* __restrict__ off, uint64_t m) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
       p += (uint64_t)gridDim.x * blockDim.x)
    rec[p].word3 = (rec[p].word3 & ~kOffMask) | (off[p] & kOffMask);
}

// ------------------------------------------------------------------------------ decode table

// Verify the exact flag of each record and derive the grid integers; a record that does not pass
// keeps the binary64 path (the definition), so a foreign or damaged header can never decode
// differently from the prediction it states.
__device__ Aux aux_of(const Record& r, uint64_t N) {
  {
    Aux a;
    a.start = r.start;
    a.A = 0;
    a.B = 0;
    bool ok = w3_exact(r.word3) && N >= 1 && N <= kMaxPartLen;
    const int s = w3_s(r.word3);
    ok = ok && s >= -11 && s <= 52;
    if (ok) {
      const double fa = r.theta0 * pow2(s), fb = r.theta1 * pow2(s);  // exact power-of-two scale
      const double lim53 = 9007199254740992.0;                        // 2^53
      ok = fa == floor(fa) && fb == floor(fb) && fabs(fa) < lim53 && fabs(fb) < lim53;
      if (ok) {
        const int64_t A = (int64_t)fa, B = (int64_t)fb;
        const i128 f0 = A, f1 = (i128)A + (i128)B * (i128)(N - 1);
        const i128 bx = (i128)B * (i128)(N - 1);
        const i128 l53 = (i128)1 << 53;
        ok = f0 < l53 && f0 > -l53 && f1 < l53 && f1 > -l53 && bx < l53 && bx > -l53;
        if (ok && s < 0) {  // scaled values must stay inside int64 (no saturation)
          const i128 g = (i128)1 << (-s);
          const i128 l63 = (i128)1 << 63;
          ok = f0 * g < l63 && f0 * g >= -l63 && f1 * g < l63 && f1 * g >= -l63;
          if (ok) {
            a.A = (int64_t)(f0 * g);
            a.B = (int64_t)((i128)B * g);
          }
        } else if (ok) {
          a.A = A;
          a.B = B;
        }
      }
    }
    a.word3 = ok ? r.word3 : (r.word3 & ~(1ull << 62));
    return a;
  }
}

// decode-table entry and polynomial table row of a polynomial partition (block pc, N values)
__device__ Aux poly_entry(const Record& r, const PolyCoef& pc, uint32_t N, PolyAux* row) {
  int32_t sj[3], S = 0;
  for (int j = 0; j < 3; j++) {
    sj[j] = (int32_t)((pc.E >> (8 * j)) & 0xFF);
    S = max(S, sj[j]);
  }
  *row = poly_aux_from(pc.K, sj, S, N);
  Aux a;
  a.A = pc.T;
  a.B = 0;
  a.start = r.start;
  a.word3 = make_w3(w3_off(r.word3) + kPolyBlockBits, w3_b(r.word3), S, 0) | kPolyFlag;
  return a;
}

__global__ void k_build_aux(const Record* __restrict__ rec, const PolyCoef* __restrict__ pcoef, uint64_t m,
                            uint64_t n, Aux* __restrict__ aux, PolyAux* __restrict__ poly) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const Record r = rec[p];
    const uint64_t e = p + 1 < m ? rec[p + 1].start : n;
    const uint64_t N = e > r.start ? e - r.start : 0;
    if (w3_poly(r.word3) && pcoef && poly)
      aux[p] = poly_entry(r, pcoef[p], (uint32_t)N, poly + p);
    else
      aux[p] = aux_of(r, N);
  }
}

// ------------------------------------------------------------------------------ packing

// Packing, one CTA per partition (staged as for the fit). Phase 1 turns each staged value into its
// zigzag residual under the partition's prediction, in shared memory (over the value itself for a
// 64-bit column, into a second region for a 32-bit one). Phase 2 has each thread assemble output
// words of the partition's bit range [off, off + N b) from those residuals. A word inside that
// range belongs to this partition alone and is stored; a word the range covers only in part holds a
// partition boundary (or the end of the stream), was zeroed beforehand, and is OR-ed into.
constexpr uint32_t kZzOffset32 = (kStageData / 2 + 32 + 127) & ~127u;  // 32-bit columns: residuals after the values
constexpr uint32_t kPackSmem64 = kStageBuf;
constexpr uint32_t kPackSmem32 = kZzOffset32 + kStageData;

// value bytes a staged partition may have: 64-bit residuals replace 64-bit values in place; a 32-bit
// column's values (up to 4096 of them) leave room for their residuals after them
__device__ __forceinline__ uint32_t pack_stage_cap(int dtype) { return dtype == LECO_U32 ? kStageData / 2 : kStageData; }

template <bool POLY>
__device__ __forceinline__ uint64_t residual_at(const Record* __restrict__ rec, const PolyAux* __restrict__ poly,
                                                const Aux& a, uint64_t p, uint32_t x, uint64_t v) {
  const int64_t pred = POLY ? predict_aux(a, rec, poly, p, x) : predict_aux_line(a, rec, p, x);
  return zz_encode((int64_t)(v - (uint64_t)pred));
}

// contribution of a 64-bit field at bit f to the output word starting at bit wb
__device__ __forceinline__ uint64_t place64(uint64_t z, uint64_t f, uint64_t wb) {
  if (f >= wb + 64 || f + 64 <= wb) return 0;
  return f >= wb ? z << (uint32_t)(f - wb) : z >> (uint32_t)(wb - f);
}

// POLY: the column may hold polynomial partitions (a separate instantiation keeps the constant and
// linear packer as small as before)
// zofs: the partition's first value within a stage holding several partitions (the 32-bit
// residual buffer is indexed like the stage). WARP: one warp packs the partition (the CTA's warps
// take different partitions of one staged item, whose residual buffers and full output words are
// disjoint), otherwise the whole CTA.
template <bool POLY, bool WARP = false>
__device__ __forceinline__ void pack_partition(const PartSrc& s, const unsigned char* st, unsigned char* ring,
                                               const Record* __restrict__ rec, const Aux* __restrict__ aux,
                                               const PolyCoef* __restrict__ pcoef, const PolyAux* __restrict__ poly,
                                               uint64_t p, uint64_t* __restrict__ words, uint32_t zofs = 0) {
  const uint32_t t = WARP ? (threadIdx.x & 31u) : threadIdx.x;
  const uint32_t G = WARP ? 32u : blockDim.x;
  auto gsync = [] {
    if (WARP)
      __syncwarp();
    else
      __syncthreads();
  };
  const Aux a = aux[p];
  const uint32_t b = w3_b(a.word3);
  const bool pl = POLY && w3_poly(a.word3) != 0;
  const uint64_t off = w3_off(a.word3), endb = off + (uint64_t)s.N * b;
  const uint64_t off0 = pl ? off - kPolyBlockBits : off;  // first bit of the partition (its block)
  if (!pl && st && b && w3_exact(a.word3)) {
    // Staged partition on the integer grid (the common case). Phase 1: each thread steps its
    // fixed-point prediction F = A + B x by B blockDim from one position to its next (no multiply).
    // Phase 2: bit positions relative to the partition's first residual bit fit 32 bits (at most
    // 2^24 fields of at most 64 bits).
    uint64_t* zs = s.dtype == LECO_U32 ? reinterpret_cast<uint64_t*>(ring + kZzOffset32) + zofs
                                       : const_cast<uint64_t*>(reinterpret_cast<const uint64_t*>(st));
    const int32_t sr = w3_s(a.word3);
    const uint32_t sh = sr > 0 ? (uint32_t)sr : 0u;
    uint64_t F = (uint64_t)a.A + (uint64_t)a.B * t;
    const uint64_t dF = (uint64_t)a.B * G;
    if (s.dtype == LECO_U32) {
      const uint32_t* v = reinterpret_cast<const uint32_t*>(st);
      for (uint32_t x = t; x < s.N; x += G, F += dF)
        zs[x] = zz_encode((int64_t)((uint64_t)v[x] - (uint64_t)((int64_t)F >> sh)));
    } else {
      const uint64_t* v = reinterpret_cast<const uint64_t*>(st);
      for (uint32_t x = t; x < s.N; x += G, F += dF)
        zs[x] = zz_encode((int64_t)(v[x] - (uint64_t)((int64_t)F >> sh)));
    }
    gsync();
    const uint32_t lead = (uint32_t)(off & 63u);
    const int32_t nbits = (int32_t)(s.N * b);
    const uint64_t w0 = off >> 6, wl = (endb - 1) >> 6;
    for (uint64_t w = w0 + t; w <= wl; w += G) {
      const int32_t r0 = (int32_t)((w - w0) << 6) - (int32_t)lead;  // the word's first bit, relative
      const int32_t r1 = r0 + 64 < nbits ? r0 + 64 : nbits;
      uint32_t x = r0 > 0 ? (uint32_t)r0 / b : 0u;
      uint64_t acc = 0;
      for (int32_t fr = (int32_t)(x * b); fr < r1; fr += (int32_t)b, x++) {
        const uint64_t z = zs[x];
        const int32_t d = fr - r0;
        acc |= d >= 0 ? z << d : z >> (-d);
      }
      if (r0 >= 0 && r0 + 64 <= nbits)
        words[w] = acc;
      else
        atomicOr((unsigned long long*)&words[w], (unsigned long long)acc);
    }
    gsync();  // the stage buffer is refilled for the next partition
    return;
  }
  if (endb > off0) {
    // phase 1: residuals into shared memory (staged partitions only; others recompute per field)
    uint64_t* zs = nullptr;
    if (st && b) {
      zs = s.dtype == LECO_U32 ? reinterpret_cast<uint64_t*>(ring + kZzOffset32) + zofs
                               : const_cast<uint64_t*>(reinterpret_cast<const uint64_t*>(st));
      if (pl) {
        // the thread's predictions T + (F(x) >> S) for x = tid, tid + blockDim, ... by forward
        // differences of the cubic F over that stride, carried times 2^(64-S) modulo 2^128 so that
        // the prediction's low 64 bits are the carried value's high half
        PolySteps Fd = poly_steps(poly[p], t, G, 64u - ((uint32_t)w3_s(a.word3) & 63u));
        const uint64_t T = (uint64_t)a.A;
        for (uint32_t xx = t; xx < s.N; xx += G) {
          zs[xx] = zz_encode((int64_t)((uint64_t)staged_value(st, s.dtype, xx) - (T + (uint64_t)(Fd.F >> 64))));
          poly_step(Fd);
        }
      } else {
        for (uint32_t x = t; x < s.N; x += G)
          zs[x] = residual_at<POLY>(rec, poly, a, p, x, (uint64_t)staged_value(st, s.dtype, x));
      }
      gsync();
    }
    // phase 2: output words of [off0, endb): the polynomial block's five words, then the fields
    for (uint64_t w = (off0 >> 6) + t; w <= ((endb - 1) >> 6); w += G) {
      const uint64_t wb = w << 6;
      const uint64_t lo = wb > off0 ? wb : off0, hi = wb + 64 < endb ? wb + 64 : endb;
      uint64_t acc = 0;
      if (pl && lo < off) {
        const PolyCoef& pc = pcoef[p];
        acc |= place64((uint64_t)pc.T, off0, wb) | place64((uint64_t)pc.K[0], off0 + 64, wb) |
               place64((uint64_t)pc.K[1], off0 + 128, wb) | place64((uint64_t)pc.K[2], off0 + 192, wb) |
               place64(pc.E, off0 + 256, wb);
      }
      if (b && hi > off) {
        const uint64_t l2 = lo > off ? lo : off;
        uint32_t x = (uint32_t)(l2 - off) / b;  // first field overlapping the word (< 2^30 bits in)
        for (uint64_t f = off + (uint64_t)x * b; f < hi; f += b, x++) {
          const uint64_t z = zs ? zs[x] : residual_at<POLY>(rec, poly, a, p, x, load_value(s.values, s.dtype, s.a + x));
          acc |= f >= wb ? z << (uint32_t)(f - wb) : z >> (uint32_t)(wb - f);
        }
      }
      if (lo == wb && hi == wb + 64)
        words[w] = acc;
      else
        atomicOr((unsigned long long*)&words[w], (unsigned long long)acc);
    }
  }
  gsync();  // the stage buffer is refilled for the next partition
}

constexpr int kPackBlock = 128;

template <bool POLY>
__global__ void __launch_bounds__(kPackBlock)
    k_pack(const void* __restrict__ values, int dtype, const Record* __restrict__ rec,
           const Aux* __restrict__ aux, const PolyCoef* __restrict__ pcoef, const PolyAux* __restrict__ poly,
           uint64_t m, uint64_t n, uint64_t* __restrict__ words, uint32_t* __restrict__ err) {
  __shared__ __align__(8) uint64_t full[1];
  extern __shared__ __align__(128) unsigned char ring[];
  auto get = [&](uint64_t p) {
    PartSrc s;
    s.values = values;
    s.n = n;
    s.a = aux[p].start;
    s.N = (uint32_t)((p + 1 < m ? aux[p + 1].start : n) - s.a);
    s.dtype = dtype;
    return s;
  };
  auto body = [&](uint64_t p, const PartSrc& s, const unsigned char* st) {
    pack_partition<POLY>(s, st, ring, rec, aux, pcoef, poly, p, words);
  };
  for_each_staged<1>(m, pack_stage_cap(dtype), get, body, ring, full, err);
}

// first stream bit of a partition: its residuals, or the block ahead of them for a polynomial one
__device__ __forceinline__ uint64_t part_first_bit(const Aux& a) {
  return w3_off(a.word3) - (w3_poly(a.word3) ? kPolyBlockBits : 0);
}

// Zero the words that packing OR-s into: each word holding a partition's first bit, and the words
// from the end of the stream on (the tail word and the zero padding). Every other word lies inside
// one partition's bit range and is written whole.
__global__ void k_zero_bounds(const Aux* __restrict__ aux, uint64_t m, uint64_t total_bits, uint64_t nwords,
                              uint64_t* __restrict__ words) {
  const uint64_t tail = total_bits >> 6;
  const uint64_t count = m + (nwords > tail ? nwords - tail : 0);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t w = i < m ? (part_first_bit(aux[i]) >> 6) : tail + (i - m);
    if (w < nwords) words[w] = 0;
  }
}

// ------------------------------------------------------------------------------ batched encode

// one warp per partition of every column (its column from the partition-column table); registers
// for 3 CTAs per SM (4 spilled, and the encode tuner then keeps 3)
__global__ void __launch_bounds__(kFitBlock, 3)
    k_fit_multi(const EncCol* __restrict__ cols, const uint64_t* __restrict__ part_base,
                const uint32_t* __restrict__ part_col, uint64_t P, int dtype, Record* __restrict__ rec,
                uint64_t* __restrict__ lenbits, uint32_t* __restrict__ max_b) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t nw = (uint64_t)gridDim.x * kFitWarps;
  for (uint64_t p = (uint64_t)blockIdx.x * kFitWarps + (threadIdx.x >> 5); p < P; p += nw) {
    const uint32_t c = part_col[p];
    const EncCol col = cols[c];
    if (col.model == LECO_MODEL_POLY) continue;  // fitted by the polynomial phases
    const uint64_t a = (p - part_base[c]) * (uint64_t)col.L;
    const uint32_t N = (uint32_t)((a + col.L < col.n ? a + col.L : col.n) - a);
    const FitResult R = fit_range<32>(col.values, dtype, a, N, col.model, lane, nullptr);
    if (lane == 0) {
      Record r;
      r.theta0 = R.theta0;
      r.theta1 = R.theta1;
      r.start = a;
      r.word3 = make_w3(0, R.b, R.s, 1);
      rec[p] = r;
      lenbits[p] = (uint64_t)N * R.b;
      if (R.b) atomicMax(max_b + c, R.b);
    }
  }
}

// column-relative offsets from the global exclusive scan, and each column's total bits
__global__ void k_set_offsets_multi(Record* __restrict__ rec, const uint64_t* __restrict__ off,
                                    const uint64_t* __restrict__ lenbits, const uint64_t* __restrict__ part_base,
                                    const uint32_t* __restrict__ part_col, uint64_t P,
                                    uint64_t* __restrict__ col_bits) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = part_col[p];
    const uint64_t base = off[part_base[c]];
    rec[p].word3 = (rec[p].word3 & ~kOffMask) | ((off[p] - base) & kOffMask);
    if (p + 1 == part_base[c + 1]) col_bits[c] = off[p] + lenbits[p] - base;
  }
}

__global__ void k_aux_multi(const Record* __restrict__ rec, const PolyCoef* __restrict__ pcoef,
                            const EncCol* __restrict__ cols, const uint64_t* __restrict__ part_base,
                            const uint32_t* __restrict__ part_col, uint64_t P, Aux* __restrict__ aux,
                            PolyAux* __restrict__ poly) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = part_col[p];
    const Record r = rec[p];
    const uint64_t e = p + 1 < part_base[c + 1] ? rec[p + 1].start : cols[c].n;
    const uint64_t N = e > r.start ? e - r.start : 0;
    if (w3_poly(r.word3) && pcoef && poly)
      aux[p] = poly_entry(r, pcoef[p], (uint32_t)N, poly + p);
    else
      aux[p] = aux_of(r, N);
  }
}

// CTA per pack item: a run of consecutive partitions of one column whose values fit one stage
// (several short partitions share one staged copy, and a warp packs each of them)
template <bool POLY>
__global__ void __launch_bounds__(kPackBlock)
    k_pack_multi(const EncCol* __restrict__ cols, const uint64_t* __restrict__ part_base,
                 const uint64_t* __restrict__ word_base, const PackItem* __restrict__ items, uint64_t nitems, int dtype,
                 const Record* __restrict__ rec, const Aux* __restrict__ aux, const PolyCoef* __restrict__ pcoef,
                 const PolyAux* __restrict__ poly, uint64_t* __restrict__ words, uint32_t* __restrict__ err) {
  __shared__ __align__(8) uint64_t full[1];
  extern __shared__ __align__(128) unsigned char ring[];
  auto get = [&](uint64_t it) {
    const PackItem item = items[it];
    const EncCol col = cols[item.c];
    const uint64_t pe = item.p0 + item.k;
    PartSrc s;
    s.values = col.values;
    s.n = col.n;
    s.a = aux[item.p0].start;
    s.N = (uint32_t)((pe < part_base[item.c + 1] ? aux[pe].start : s.n) - s.a);
    s.dtype = dtype;
    return s;
  };
  auto body = [&](uint64_t it, const PartSrc& si, const unsigned char* st) {
    const PackItem item = items[it];
    const uint64_t p0 = part_base[item.c];
    const uint32_t vb = dtype == LECO_U32 ? 4u : 8u;
    auto part = [&](uint64_t p) {
      PartSrc s = si;
      s.a = aux[p].start;
      s.N = (uint32_t)((p + 1 < part_base[item.c + 1] ? aux[p + 1].start : si.n) - s.a);
      return s;
    };
    if (item.k == 1) {  // one partition: the whole CTA
      pack_partition<POLY>(part(item.p0), st, ring, rec + p0, aux + p0, POLY ? pcoef + p0 : nullptr,
                           POLY ? poly + p0 : nullptr, item.p0 - p0, words + word_base[item.c], 0);
      return;
    }
    // several short partitions: a warp each, the CTA's warps side by side (their residual buffers
    // and whole output words are disjoint)
    for (uint32_t q = threadIdx.x >> 5; q < item.k; q += kPackBlock / 32) {
      const uint64_t p = item.p0 + q;
      const PartSrc s = part(p);
      const uint32_t zofs = (uint32_t)(s.a - si.a);
      pack_partition<POLY, true>(s, st ? st + (size_t)zofs * vb : nullptr, ring, rec + p0, aux + p0,
                                 POLY ? pcoef + p0 : nullptr, POLY ? poly + p0 : nullptr, p - p0,
                                 words + word_base[item.c], zofs);
    }
    __syncthreads();  // the stage buffer is refilled for the next item
  };
  for_each_staged<1>(nitems, pack_stage_cap(dtype), get, body, ring, full, err);
}

// Pack items of one column with short partitions (variable partitions): a partition of at most
// kItemWindow values joins the item of its predecessor when both start in the same kItemWindow-aligned
// window of positions (so an item spans fewer than 2 kItemWindow values and fits one stage); a longer
// partition is an item of its own. flag[p] = 1 where an item begins.
constexpr uint64_t kItemWindow = 2048;

__global__ void k_item_flags(const Aux* __restrict__ aux, uint64_t m, uint64_t n, uint64_t* __restrict__ flag) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = aux[p].start, e = p + 1 < m ? aux[p + 1].start : n;
    bool begin = p == 0 || e - s > kItemWindow;
    if (!begin) {
      const uint64_t s0 = aux[p - 1].start;
      begin = s - s0 > kItemWindow || (s / kItemWindow) != (s0 / kItemWindow);
    }
    flag[p] = begin ? 1ull : 0ull;
  }
}

// item_start[idx[p]] = p for every item-beginning partition p, and item_start[nitems] = m
__global__ void k_item_starts(const uint64_t* __restrict__ flag, const uint64_t* __restrict__ idx, uint64_t m,
                              const uint64_t* __restrict__ nitems, uint64_t* __restrict__ item_start) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m; p += (uint64_t)gridDim.x * blockDim.x) {
    if (flag[p]) item_start[idx[p]] = p;
    if (p == 0) item_start[*nitems] = m;
  }
}

// CTA per item of one column (constant and linear partitions): one staged copy for the item's
// partitions, packed one after the other; the item count is read on the device
__global__ void __launch_bounds__(kPackBlock)
    k_pack_items(const void* __restrict__ values, int dtype, const Record* __restrict__ rec,
                 const Aux* __restrict__ aux, uint64_t m, uint64_t n, const uint64_t* __restrict__ item_start,
                 const uint64_t* __restrict__ nitems_d, uint64_t* __restrict__ words, uint32_t* __restrict__ err) {
  __shared__ __align__(8) uint64_t full[1];
  extern __shared__ __align__(128) unsigned char ring[];
  const uint64_t nitems = *nitems_d;
  auto get = [&](uint64_t it) {
    const uint64_t p0 = item_start[it], pe = item_start[it + 1];
    PartSrc s;
    s.values = values;
    s.n = n;
    s.a = aux[p0].start;
    s.N = (uint32_t)((pe < m ? aux[pe].start : n) - s.a);
    s.dtype = dtype;
    return s;
  };
  auto body = [&](uint64_t it, const PartSrc& si, const unsigned char* st) {
    const uint64_t p0 = item_start[it], pe = item_start[it + 1];
    const uint32_t vb = dtype == LECO_U32 ? 4u : 8u;
    auto part = [&](uint64_t p) {
      PartSrc s = si;
      s.a = aux[p].start;
      s.N = (uint32_t)((p + 1 < m ? aux[p + 1].start : n) - s.a);
      return s;
    };
    if (pe - p0 == 1) {  // a long partition: the whole CTA
      pack_partition<false>(part(p0), st, ring, rec, aux, nullptr, nullptr, p0, words, 0);
      return;
    }
    // short partitions: a warp each, the CTA's warps side by side
    for (uint64_t p = p0 + (threadIdx.x >> 5); p < pe; p += kPackBlock / 32) {
      const PartSrc s = part(p);
      const uint32_t zofs = (uint32_t)(s.a - si.a);
      pack_partition<false, true>(s, st ? st + (size_t)zofs * vb : nullptr, ring, rec, aux, nullptr, nullptr, p, words,
                                  zofs);
    }
    __syncthreads();  // the stage buffer is refilled for the next item
  };
  for_each_staged<1>(nitems, pack_stage_cap(dtype), get, body, ring, full, err);
}

__global__ void k_part_col(const uint64_t* __restrict__ part_base, uint32_t ncols, uint64_t P,
                           uint32_t* __restrict__ part_col) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x)
    part_col[p] = find_col(part_base, ncols, p);
}

// exclusive prefix sum of the columns' stream words: each thread sums a contiguous run of columns,
// the CTA scans the run totals, then each thread writes its run's bases
constexpr int kWordBaseBlock = 1024;
__global__ void __launch_bounds__(kWordBaseBlock)
    k_word_bases(const uint64_t* __restrict__ col_bits, uint32_t ncols, uint64_t* __restrict__ word_base) {
  __shared__ uint64_t run[kWordBaseBlock];
  const uint32_t t = threadIdx.x;
  const uint64_t per = ((uint64_t)ncols + kWordBaseBlock - 1) / kWordBaseBlock;
  const uint32_t c0 = (uint32_t)min((uint64_t)t * per, (uint64_t)ncols);
  const uint32_t c1 = (uint32_t)min((uint64_t)c0 + per, (uint64_t)ncols);
  uint64_t s = 0;
  for (uint32_t c = c0; c < c1; c++) s += stream_words(col_bits[c]);
  run[t] = s;
  __syncthreads();
  for (uint32_t d = 1; d < kWordBaseBlock; d <<= 1) {
    const uint64_t add = t >= d ? run[t - d] : 0;
    __syncthreads();
    run[t] += add;
    __syncthreads();
  }
  uint64_t base = run[t] - s;
  for (uint32_t c = c0; c < c1; c++) {
    word_base[c] = base;
    base += stream_words(col_bits[c]);
  }
  if (t == kWordBaseBlock - 1) word_base[ncols] = run[t];
}

// k_zero_bounds for every column: thread per partition, then each column's tail words
__global__ void k_zero_bounds_multi(const Aux* __restrict__ aux, const uint32_t* __restrict__ part_col,
                                    const uint64_t* __restrict__ word_base, const uint64_t* __restrict__ col_bits,
                                    uint32_t ncols, uint64_t P, uint64_t* __restrict__ words) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P; p += stride) {
    const uint32_t c = part_col[p];
    words[word_base[c] + (part_first_bit(aux[p]) >> 6)] = 0;
  }
  for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < ncols; c += stride)
    for (uint64_t w = word_base[c] + (col_bits[c] >> 6); w < word_base[c + 1]; w++) words[w] = 0;
}

int grid_for(uint64_t items, int per_block, int max_blocks_per_sm) {
  const uint64_t need = (items + per_block - 1) / per_block;
  const uint64_t cap = (uint64_t)sm_count() * max_blocks_per_sm;
  return (int)(need < cap ? (need ? need : 1) : cap);
}

}  // namespace

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = v > 0 ? v : 1;
  }
  return cached[dev];
}

// persistent grid: as many CTAs as fit on the GPU at once with the staging ring (grid-stride over work)
template <typename K>
int resident_grid(K kern, int block, uint64_t work, uint32_t smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, block, smem) != cudaSuccess || nb < 1) nb = 1;
  const uint64_t cap = (uint64_t)sm_count() * nb;
  return (int)(work < cap ? work : cap);
}

// the four polynomial phases over partitions [0, m) of the map, with their scratch (given: at least
// poly_fit_scratch_bytes(m) bytes the caller owns; nullptr: taken from the pool and released)
template <typename Map>
cudaError_t launch_poly_fit(const Map& map, int dtype, uint64_t m, Record* rec, uint64_t* lenbits, PolyCoef* pcoef,
                            uint32_t* max_b, cudaStream_t st, void* given = nullptr) {
  const uint64_t bm = (sizeof(PolyMom) * m + 255) & ~255ull, bp = (sizeof(PolyPlan) * m + 255) & ~255ull;
  char* scr = static_cast<char*>(given);
  cudaError_t e = given ? cudaSuccess : dev_alloc((void**)&scr, bm + bp + sizeof(PolyRange) * m, st);
  if (e != cudaSuccess) return e;
  PolyMom* mom = reinterpret_cast<PolyMom*>(scr);
  PolyPlan* plan = reinterpret_cast<PolyPlan*>(scr + bm);
  PolyRange* rng = reinterpret_cast<PolyRange*>(scr + bm + bp);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_poly_ranges<Map>, kFitBlock, 0) != cudaSuccess || nb < 1)
    nb = 1;
  const uint64_t wb = (m + kFitWarps - 1) / kFitWarps;
  k_poly_moments<Map><<<grid_for(wb, 1, 8), kFitBlock, 0, st>>>(map, dtype, m, mom);
  k_poly_plan<Map><<<grid_for(m, 128, 8), 128, 0, st>>>(map, m, mom, plan);
  k_poly_ranges<Map><<<grid_for(wb, 1, nb), kFitBlock, 0, st>>>(map, dtype, m, plan, rng);
  k_poly_choose<Map><<<grid_for(m, 128, 8), 128, 0, st>>>(map, m, mom, plan, rng, rec, lenbits, pcoef, max_b);
  e = cudaGetLastError();
  if (!given) cudaFreeAsync(scr, st);
  return e;
}

cudaError_t launch_fit(const void* values, int dtype, uint64_t n, const uint64_t* starts,
                       uint32_t L, uint64_t m, int model, Record* rec, uint64_t* lenbits, PolyCoef* pcoef,
                       uint32_t* max_b, uint32_t* err, cudaStream_t st) {
  (void)err;  // the fit waits on nothing
  if (model == LECO_MODEL_POLY && !pcoef) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(max_b, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess || m == 0) return e;
  if (model == LECO_MODEL_POLY) return launch_poly_fit(OneColumn{values, n, starts, L}, dtype, m, rec, lenbits, pcoef,
                                                        max_b, st);
  // fit CTAs per SM: the encode shape of the tuning table for this value width (fewer keep more of
  // each partition in L2 between the two passes)
  const uint32_t fc = encode_config_lookup(dtype).fit_ctas;
  const int ctas = fc >= 1 && fc <= (uint32_t)kFitCtasPerSm ? (int)fc : kFitCtasPerSm;
  // partitions of at least 1024 values: two warps each (the second pass then stays in L2)
  if (!starts && L >= 1024) {
    k_fit_pairs<<<grid_for((m + kFitPairs - 1) / kFitPairs, 1, ctas), kFitBlock, 0, st>>>(values, dtype, n, starts,
                                                                                        L, m, model, rec, lenbits,
                                                                                        max_b);
    return cudaGetLastError();
  }
  k_fit<<<grid_for((m + kFitWarps - 1) / kFitWarps, 1, ctas), kFitBlock, 0, st>>>(values, dtype, n, starts, L, m,
                                                                                  model, rec, lenbits, max_b);
  return cudaGetLastError();
}

uint64_t offsets_scratch_elems(uint64_t m) {
  const uint64_t ntiles = (m + kPrefixTile - 1) / kPrefixTile;
  return m + ntiles + 1;  // exclusive offsets + tile prefixes + total
}

// exclusive scan of in[0..count) into out; *total (device) = the sum. scratch: ntiles+1 elems.
cudaError_t scan_u64(const uint64_t* in, uint64_t count, uint64_t* out, uint64_t* scratch,
                     uint64_t* total, cudaStream_t st) {
  if (count == 0) return cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
  const uint64_t ntiles = (count + kPrefixTile - 1) / kPrefixTile;
  k_prefix_tiles<<<(unsigned)ntiles, kPrefixBlock, 0, st>>>(in, count, scratch);
  k_prefix_top<<<1, kPrefixBlock, 0, st>>>(scratch, ntiles, total);
  k_prefix_apply<<<(unsigned)ntiles, kPrefixBlock, 0, st>>>(in, count, scratch, out);
  return cudaGetLastError();
}

cudaError_t launch_offsets(Record* rec, const uint64_t* lenbits, uint64_t m, uint64_t* scratch,
                           uint64_t scratch_elems, uint64_t* total_out, cudaStream_t st) {
  (void)scratch_elems;
  if (m == 0) return cudaMemsetAsync(total_out, 0, sizeof(uint64_t), st);
  uint64_t* off = scratch;
  uint64_t* tiles = scratch + m;
  cudaError_t e = scan_u64(lenbits, m, off, tiles, total_out, st);
  if (e != cudaSuccess) return e;
  k_set_offsets<<<grid_for(m, 256, 8), 256, 0, st>>>(rec, off, m);
  return cudaGetLastError();
}

cudaError_t launch_build_aux(const Record* rec, const PolyCoef* pcoef, uint64_t m, uint64_t n, Aux* aux,
                             PolyAux* poly, uint32_t* status, cudaStream_t st) {
  (void)status;
  if (m == 0) return cudaSuccess;
  k_build_aux<<<grid_for(m, 256, 8), 256, 0, st>>>(rec, pcoef, m, n, aux, poly);
  return cudaGetLastError();
}

cudaError_t launch_pack(const void* values, int dtype, const Record* rec, const Aux* aux, const PolyCoef* pcoef,
                        const PolyAux* poly, uint64_t m, uint64_t n, uint64_t total_bits, uint64_t* words,
                        uint64_t nwords, uint32_t* err, cudaStream_t st) {
  if (nwords == 0) return cudaSuccess;
  const uint64_t tail = total_bits >> 6;
  k_zero_bounds<<<grid_for(m + (nwords > tail ? nwords - tail : 0), 256, 8), 256, 0, st>>>(aux, m, total_bits, nwords,
                                                                                         words);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || m == 0) return e;
  const uint32_t smem = dtype == LECO_U32 ? kPackSmem32 : kPackSmem64;
  if (pcoef)
    k_pack<true><<<resident_grid(k_pack<true>, kPackBlock, m, smem), kPackBlock, smem, st>>>(
        values, dtype, rec, aux, pcoef, poly, m, n, words, err);
  else
    k_pack<false><<<resident_grid(k_pack<false>, kPackBlock, m, smem), kPackBlock, smem, st>>>(
        values, dtype, rec, aux, nullptr, nullptr, m, n, words, err);
  return cudaGetLastError();
}

cudaError_t launch_pack_var(const void* values, int dtype, const Record* rec, const Aux* aux, uint64_t m, uint64_t n,
                            uint64_t total_bits, uint64_t* words, uint64_t nwords, uint32_t* err, cudaStream_t st) {
  if (nwords == 0) return cudaSuccess;
  const uint64_t tail = total_bits >> 6;
  k_zero_bounds<<<grid_for(m + (nwords > tail ? nwords - tail : 0), 256, 8), 256, 0, st>>>(aux, m, total_bits, nwords,
                                                                                         words);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || m == 0) return e;
  // flags | indices | item starts (m + 1) | scan scratch | item count
  const uint64_t scr_elems = m / 2048 + 2;
  uint64_t* buf = nullptr;
  e = dev_alloc((void**)&buf, 8 * (3 * m + 1 + scr_elems + 2), st);
  if (e != cudaSuccess) return e;
  uint64_t* flag = buf;
  uint64_t* idx = buf + m;
  uint64_t* item_start = buf + 2 * m;
  uint64_t* scr = item_start + m + 1;
  uint64_t* nitems = scr + scr_elems + 1;
  k_item_flags<<<grid_for(m, 256, 8), 256, 0, st>>>(aux, m, n, flag);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = scan_u64(flag, m, idx, scr, nitems, st);
  if (e == cudaSuccess) {
    k_item_starts<<<grid_for(m, 256, 8), 256, 0, st>>>(flag, idx, m, nitems, item_start);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const uint32_t smem = dtype == LECO_U32 ? kPackSmem32 : kPackSmem64;
    // every item holds at least one partition: m bounds the count the grid is sized for
    k_pack_items<<<resident_grid(k_pack_items, kPackBlock, m, smem), kPackBlock, smem, st>>>(
        values, dtype, rec, aux, m, n, item_start, nitems, words, err);
    e = cudaGetLastError();
  }
  cudaFreeAsync(buf, st);
  return e;
}

cudaError_t launch_part_col(const uint64_t* part_base, uint32_t ncols, uint64_t P, uint32_t* part_col, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  k_part_col<<<grid_for(P, 256, 8), 256, 0, st>>>(part_base, ncols, P, part_col);
  return cudaGetLastError();
}

uint64_t poly_fit_scratch_bytes(uint64_t m) {
  return ((sizeof(PolyMom) * m + 255) & ~255ull) + ((sizeof(PolyPlan) * m + 255) & ~255ull) + sizeof(PolyRange) * m;
}

cudaError_t launch_fit_multi(const EncCol* cols, const uint64_t* part_base, const uint32_t* part_col, uint32_t ncols,
                             uint64_t P, int dtype, Record* rec, uint64_t* lenbits, PolyCoef* pcoef, uint32_t* max_b,
                             uint32_t* err, uint32_t fit_ctas, cudaStream_t st, void* poly_scratch) {
  (void)err;
  cudaError_t e = cudaMemsetAsync(max_b, 0, sizeof(uint32_t) * (ncols ? ncols : 1), st);
  if (e != cudaSuccess || P == 0) return e;
  const int ctas = fit_ctas >= 1 && fit_ctas <= (uint32_t)kFitCtasPerSm ? (int)fit_ctas : kFitCtasPerSm;
  const int grid = grid_for((P + kFitWarps - 1) / kFitWarps, 1, ctas);
  k_fit_multi<<<grid, kFitBlock, 0, st>>>(cols, part_base, part_col, P, dtype, rec, lenbits, max_b);
  e = cudaGetLastError();
  if (e == cudaSuccess && pcoef)
    e = launch_poly_fit(BatchColumns{cols, part_base, ncols}, dtype, P, rec, lenbits, pcoef, max_b, st, poly_scratch);
  return e;
}

uint64_t offsets_multi_scratch_elems(uint64_t P) { return P + (P + kPrefixTile - 1) / kPrefixTile + 2; }

cudaError_t launch_offsets_multi(Record* rec, const uint64_t* lenbits, const uint64_t* part_base,
                                 const uint32_t* part_col, uint32_t ncols, uint64_t P, uint64_t* scratch,
                                 uint64_t* col_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(col_bits, 0, sizeof(uint64_t) * (ncols ? ncols : 1), st);
  if (e != cudaSuccess || P == 0) return e;
  uint64_t* off = scratch;
  uint64_t* tiles = scratch + P;
  uint64_t* total = scratch + offsets_multi_scratch_elems(P) - 1;
  e = scan_u64(lenbits, P, off, tiles, total, st);
  if (e != cudaSuccess) return e;
  k_set_offsets_multi<<<grid_for(P, 256, 8), 256, 0, st>>>(rec, off, lenbits, part_base, part_col, P, col_bits);
  return cudaGetLastError();
}

cudaError_t launch_aux_multi(const Record* rec, const PolyCoef* pcoef, const EncCol* cols, const uint64_t* part_base,
                             const uint32_t* part_col, uint64_t P, Aux* aux, PolyAux* poly, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  k_aux_multi<<<grid_for(P, 256, 8), 256, 0, st>>>(rec, pcoef, cols, part_base, part_col, P, aux, poly);
  return cudaGetLastError();
}

uint32_t pack_item_values() { return kStageData / 8; }

cudaError_t launch_word_bases(const uint64_t* col_bits, uint32_t ncols, uint64_t* word_base, cudaStream_t st) {
  k_word_bases<<<1, kWordBaseBlock, 0, st>>>(col_bits, ncols, word_base);
  return cudaGetLastError();
}

cudaError_t launch_pack_multi(const EncCol* cols, const uint64_t* part_base, const uint32_t* part_col,
                              const uint64_t* word_base, const uint64_t* col_bits, const PackItem* items,
                              uint64_t nitems, uint32_t ncols, uint64_t P, uint64_t W, int dtype, const Record* rec,
                              const Aux* aux, const PolyCoef* pcoef, const PolyAux* poly, uint64_t* words,
                              uint32_t* err, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  k_zero_bounds_multi<<<grid_for(P > ncols ? P : ncols, 256, 8), 256, 0, st>>>(aux, part_col, word_base, col_bits,
                                                                                ncols, P, words);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nitems == 0) return e;
  const uint32_t smem = dtype == LECO_U32 ? kPackSmem32 : kPackSmem64;
  if (pcoef)
    k_pack_multi<true><<<resident_grid(k_pack_multi<true>, kPackBlock, nitems, smem), kPackBlock, smem, st>>>(
        cols, part_base, word_base, items, nitems, dtype, rec, aux, pcoef, poly, words, err);
  else
    k_pack_multi<false><<<resident_grid(k_pack_multi<false>, kPackBlock, nitems, smem), kPackBlock, smem, st>>>(
        cols, part_base, word_base, items, nitems, dtype, rec, aux, nullptr, nullptr, words, err);
  return cudaGetLastError();
}

}  // namespace leco
