// Internal definitions of the GB300 LeCo library: device layouts, format accessors and the
// device helpers shared by the kernels. Not part of the public ABI (see include/leco.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "leco.h"

namespace leco {

typedef __int128 i128;
typedef unsigned __int128 u128;

constexpr uint64_t kOffMask = (1ull << 48) - 1;
constexpr uint32_t kMaxPartLen = 1u << 24;  // keeps every fit quantity inside int128
constexpr uint64_t kSmBits = 256;           // model size S_M: one 32-byte record (§3.2.2)

// Canonical 32-byte partition header (§3.3 storage format): theta as binary64.
struct Record {
  double theta0;
  double theta1;
  uint64_t start;
  uint64_t word3;  // off:48 | b:7 | s:7 | exact:1 | poly:1
};
static_assert(sizeof(Record) == 32, "record layout");

// Device decode table, derived from the records when a column is created: the same header with
// theta replaced by the grid integers (A, B) when the exact flag was verified. word3 keeps the
// canonical layout; its exact bit is cleared when verification failed (binary64 path then).
// A polynomial partition's entry has A = T, B = 0, the poly bit, exact = 0, s = the common grid
// exponent S of its coefficients and off moved past its coefficient block to its first residual;
// its prediction comes from the PolyAux table.
struct Aux {
  int64_t A;
  int64_t B;
  uint64_t start;
  uint64_t word3;
};
static_assert(sizeof(Aux) == 32, "aux layout");

// Polynomial model (§3.1; §4's per-partition choice among constant, linear and polynomials up to
// degree three). A polynomial partition's stream bits begin with a block of five 64-bit words
// {T, K1, K2, K3, E = s1 | s2 << 8 | s3 << 16}; its prediction is
// T + floor(sum_j K_j p_j(x) 2^-s_j) mod 2^64 over the Gram polynomials of its N values on
// x' = 2x - (N-1): p1 = x', p2 = 3x'^2 - (N^2-1), p3 = 5x'^3 - (3N^2-7)x'.
constexpr uint32_t kPolyBlockBits = 320;
constexpr uint32_t kPolyMinLen = 64;
constexpr uint32_t kPolyMaxLen = 16384;
// extra staged bytes a scan tile can need for the blocks of polynomial partitions that start
// inside it (at most kScanTile / kPolyMinLen of them)
constexpr uint32_t kPolyStageExtra = 4096 / kPolyMinLen * (kPolyBlockBits / 8);

// the block as the encoder writes it (one per partition; used only for polynomial partitions)
struct PolyCoef {
  int64_t T;
  int64_t K[3];
  uint64_t E;
};
static_assert(sizeof(PolyCoef) == 40, "poly coefficient layout");

// Decode-side form: F(x) = a0 + a1 x + a2 x^2 + a3 x^3 = sum_j K_j 2^(S - s_j) p_j(x) expanded in
// the local index (exact 128-bit integers), so that pred(x) = T + (F(x) >> S).
struct PolyAux {
  uint64_t a[4][2];  // a_k as (low, high) 64-bit halves of a two's complement 128-bit integer
};
static_assert(sizeof(PolyAux) == 64, "poly aux layout");

// Scan tiles: tile t covers positions [t kScanTile, (t+1) kScanTile). Positions are encoded in order
// with dense bit offsets, so a tile's residuals are one contiguous bit range; its descriptor is
// built once per column and names the 16-byte-aligned word range to stage and the tile's value
// bounds under the models (used to skip groups and, with pruning, whole tiles).
constexpr uint64_t kScanTile = 4096;

struct TileDesc {
  uint64_t p0;      // first partition touching the tile
  uint64_t g0;      // byte offset of the staged word range in the residual stream (16-aligned)
  uint64_t vmin;    // bounds == 1: every value of the tile lies in [vmin, vmax] (unsigned);
  uint64_t vmax;    // bounds == 2: in [0, vmax] or [vmin, 2^64 - 1] (vmax < vmin); 0: unknown
  uint32_t np;      // partitions touching the tile
  uint32_t wbytes;  // bytes of the staged word range (multiple of 16)
  uint32_t bounds;
  uint32_t pad;
};
static_assert(sizeof(TileDesc) == 48, "tile descriptor layout");

__host__ __device__ __forceinline__ uint64_t scan_tiles(uint64_t n) { return (n + kScanTile - 1) / kScanTile; }

// shared-memory bytes of one staged word range when no partition is wider than max_b bits
__host__ __device__ __forceinline__ uint32_t stage_word_bytes(uint32_t max_b) {
  const uint64_t bytes = kScanTile * (uint64_t)max_b / 8 + 64;
  return (uint32_t)((bytes + 15) & ~15ull);
}

// status word bits (device)
enum : uint32_t { kStatIndexRange = 1u, kStatCorrupt = 2u, kStatTimeout = 4u };

__host__ __device__ __forceinline__ uint64_t w3_off(uint64_t w3) { return w3 & kOffMask; }
__host__ __device__ __forceinline__ uint32_t w3_b(uint64_t w3) { return (uint32_t)(w3 >> 48) & 0x7Fu; }
__host__ __device__ __forceinline__ int32_t w3_s(uint64_t w3) {
  int32_t s = (int32_t)((w3 >> 55) & 0x7F);
  return s >= 64 ? s - 128 : s;
}
__host__ __device__ __forceinline__ uint32_t w3_exact(uint64_t w3) { return (uint32_t)(w3 >> 62) & 1u; }
__host__ __device__ __forceinline__ uint32_t w3_poly(uint64_t w3) { return (uint32_t)(w3 >> 63); }
constexpr uint64_t kPolyFlag = 1ull << 63;
__host__ __device__ __forceinline__ uint64_t make_w3(uint64_t off, uint32_t b, int32_t s, uint32_t exact) {
  return (off & kOffMask) | ((uint64_t)(b & 0x7F) << 48) | ((uint64_t)((uint32_t)s & 0x7F) << 55) |
         ((uint64_t)(exact & 1) << 62);
}

// words a stream of total_bits needs: data words + 2 zero padding words, rounded up to 16 bytes
__host__ __device__ __forceinline__ uint64_t stream_words(uint64_t total_bits) {
  uint64_t w = (total_bits + 63) / 64 + 2;
  return (w + 1) & ~1ull;
}

// ---------------------------------------------------------------------------- device helpers

__device__ __forceinline__ uint64_t zz_encode(int64_t r) {
  return ((uint64_t)r << 1) ^ (uint64_t)(r >> 63);
}
__device__ __forceinline__ int64_t zz_decode(uint64_t z) {
  return (int64_t)((z >> 1) ^ (0ull - (z & 1ull)));
}
__device__ __forceinline__ uint64_t low_mask(uint32_t b) {
  return b >= 64 ? ~0ull : ((1ull << b) - 1ull);
}

// b-bit field at absolute bit position pos of the LSB-first stream. The stream's padding words
// make words[pos/64 + 1] readable for every pos <= total bits.
__device__ __forceinline__ uint64_t read_field(const uint64_t* __restrict__ words, uint64_t pos,
                                               uint32_t b) {
  const uint64_t w = pos >> 6;
  const uint32_t o = (uint32_t)pos & 63u;
  const uint64_t lo = __ldg(words + w);
  const uint64_t hi = __ldg(words + w + 1);
  // (hi << 1) << (63 - o) is hi << (64 - o) without the undefined shift by 64 when o == 0
  return ((lo >> o) | ((hi << 1) << (63 - o))) & low_mask(b);
}

// binary64 prediction of §3.3: floor(fl(fl(theta1 * x) + theta0)), NaN -> 0, saturating
__device__ __forceinline__ int64_t predict_f64(double theta0, double theta1, uint64_t x) {
  const double y = __dadd_rn(__dmul_rn(theta1, __ull2double_rn(x)), theta0);
  if (y != y) return 0;
  if (y >= 9223372036854775808.0) return INT64_MAX;
  if (y < -9223372036854775808.0) return INT64_MIN;
  return __double2ll_rd(y);
}

// F(x) of a polynomial partition by Horner's rule in 128-bit two's complement arithmetic (exact:
// the true F is below 2^126 in magnitude, so wrap-around in the intermediate steps cancels)
__device__ __forceinline__ i128 poly_eval(const PolyAux* __restrict__ poly, uint64_t p, uint64_t x) {
  const ulonglong2* q = reinterpret_cast<const ulonglong2*>(poly + p);
  const ulonglong2 c0 = __ldg(q), c1 = __ldg(q + 1), c2 = __ldg(q + 2), c3 = __ldg(q + 3);
  const u128 X = x;
  u128 F = ((u128)c3.y << 64) | c3.x;
  F = F * X + (((u128)c2.y << 64) | c2.x);
  F = F * X + (((u128)c1.y << 64) | c1.x);
  F = F * X + (((u128)c0.y << 64) | c0.x);
  return (i128)F;
}

// prediction of a constant or linear partition from the decode table (integer grid when exact,
// else binary64 from the record)
__device__ __forceinline__ int64_t predict_aux_line(const Aux& a, const Record* __restrict__ rec, uint64_t p,
                                                    uint64_t x) {
  if (w3_exact(a.word3)) {
    const int32_t s = w3_s(a.word3);
    const int64_t f = a.A + a.B * (int64_t)x;
    return s > 0 ? (f >> s) : f;
  }
  return predict_f64(__ldg(&rec[p].theta0), __ldg(&rec[p].theta1), x);
}

// prediction of any partition (the polynomial table for a polynomial one)
__device__ __forceinline__ int64_t predict_aux(const Aux& a, const Record* __restrict__ rec,
                                               const PolyAux* __restrict__ poly, uint64_t p, uint64_t x) {
  if (w3_poly(a.word3)) return (int64_t)((uint64_t)a.A + (uint64_t)(poly_eval(poly, p, x) >> w3_s(a.word3)));
  return predict_aux_line(a, rec, p, x);
}

__device__ __forceinline__ uint64_t load_value(const void* __restrict__ v, int dtype, uint64_t i) {
  return dtype == LECO_U32 ? (uint64_t)__ldg((const uint32_t*)v + i) : __ldg((const uint64_t*)v + i);
}

__device__ __forceinline__ int bitlen_u64(uint64_t x) { return 64 - __clzll((long long)x); }
// exact 128-bit products from 64-bit multiplies (the generic 128 x 128-bit product is not needed
// when one factor has 64 bits): a * b for int64 a, b; a * b mod 2^128 for a 128-bit a, unsigned b
__device__ __forceinline__ i128 mul_s64(int64_t a, int64_t b) {
  return (i128)(((u128)(uint64_t)__mul64hi(a, b) << 64) | (u128)((uint64_t)a * (uint64_t)b));
}
__device__ __forceinline__ i128 mul_i128_u64(i128 a, uint64_t b) {
  const uint64_t al = (uint64_t)a, ah = (uint64_t)((u128)a >> 64);
  return (i128)(((u128)(__umul64hi(al, b) + ah * b) << 64) | (u128)(al * b));
}

__device__ __forceinline__ int bitlen_u128(u128 x) {
  const uint64_t hi = (uint64_t)(x >> 64);
  return hi ? 128 - __clzll((long long)hi) : bitlen_u64((uint64_t)x);
}

// SplitMix64 (Steele, Lea & Flood 2014): first output of the generator seeded with x
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// warp reductions
__device__ __forceinline__ i128 warp_sum_i128(i128 v) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)((u128)v >> 64);
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t l2 = __shfl_down_sync(0xffffffffu, lo, o);
    const uint64_t h2 = __shfl_down_sync(0xffffffffu, hi, o);
    const uint64_t nl = lo + l2;
    hi = hi + h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  return (i128)(((u128)hi << 64) | lo);
}
__device__ __forceinline__ int64_t warp_max_i64(int64_t v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, (int64_t)__shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int64_t warp_min_i64(int64_t v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, (int64_t)__shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, (uint64_t)__shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------- host-side launchers
// (defined in the .cu files; all return cudaError_t of the launch)

struct ColumnView {
  uint64_t n;
  uint64_t m;
  int dtype;
  uint32_t L;                  // fixed partition length, 0 for variable
  const Record* rec;
  const Aux* aux;
  const uint64_t* words;
  const uint64_t* starts;      // variable: m+1 entries; fixed: nullptr
  const TileDesc* tiles;       // scan_tiles(n) descriptors
  const PolyAux* poly;         // m entries when the column may hold polynomial partitions, else nullptr
  uint32_t stage_bytes;        // stage_word_bytes(max width of the column)
  uint32_t* status;
};

// Tunable shape of the scan pipeline: shared-memory stages in flight per CTA and consumer warps.
struct ScanConfig {
  uint32_t stages;
  uint32_t consumer_warps;
};

// One job of a multi-column scan: positions [begin, end) of scan tile `tile` of column `col`,
// decoded to out (position i -> out[i - begin]).
struct BatchItem {
  uint32_t col;
  uint32_t pad;
  uint64_t tile;
  uint64_t begin;
  uint64_t end;
  void* out;
};
static_assert(sizeof(BatchItem) == 40, "batch item layout");

// One column of a batched encode (fixed partitions of length L).
struct EncCol {
  const void* values;
  uint64_t n;
  uint32_t L;
  int32_t model;
};

// batched encode (k_encode.cu, k_scan.cu): arrays of all columns back to back; part_base /
// word_base / tile_base hold each column's first partition / word / scan tile (ncols + 1 entries)
// pcoef / poly: as for one column, over all P partitions (nullptr when no column takes the
// polynomial model; a polynomial column's partitions are fitted by the polynomial phases)
// part_col[p]: the column of global partition p (launch_part_col fills it once per batch)
cudaError_t launch_part_col(const uint64_t* part_base, uint32_t ncols, uint64_t P, uint32_t* part_col, cudaStream_t st);
// poly_scratch: poly_fit_scratch_bytes(P) caller-owned bytes for the polynomial phases, or nullptr
// (then taken from the library pool for the call)
uint64_t poly_fit_scratch_bytes(uint64_t m);
cudaError_t launch_fit_multi(const EncCol* cols, const uint64_t* part_base, const uint32_t* part_col, uint32_t ncols,
                             uint64_t P, int dtype, Record* rec, uint64_t* lenbits, PolyCoef* pcoef, uint32_t* max_b,
                             uint32_t* err, uint32_t fit_ctas, cudaStream_t st, void* poly_scratch = nullptr);
uint64_t offsets_multi_scratch_elems(uint64_t P);
cudaError_t launch_offsets_multi(Record* rec, const uint64_t* lenbits, const uint64_t* part_base,
                                 const uint32_t* part_col, uint32_t ncols, uint64_t P, uint64_t* scratch,
                                 uint64_t* col_bits, cudaStream_t st);
cudaError_t launch_aux_multi(const Record* rec, const PolyCoef* pcoef, const EncCol* cols, const uint64_t* part_base,
                             const uint32_t* part_col, uint64_t P, Aux* aux, PolyAux* poly, cudaStream_t st);
// A pack item: k consecutive partitions p0 .. p0 + k - 1 (global indices) of column c, packed by one
// CTA from one staged copy; at most pack_item_values() values, one partition for polynomial columns.
struct PackItem {
  uint64_t p0;
  uint32_t c;
  uint32_t k;
};
uint32_t pack_item_values();
// word_base[c] = sum of stream_words(col_bits[k]) over k < c, for c = 0 .. ncols, on the device (one
// CTA): each column's packed stream placed right after the previous one
cudaError_t launch_word_bases(const uint64_t* col_bits, uint32_t ncols, uint64_t* word_base, cudaStream_t st);
cudaError_t launch_pack_multi(const EncCol* cols, const uint64_t* part_base, const uint32_t* part_col,
                              const uint64_t* word_base, const uint64_t* col_bits, const PackItem* items,
                              uint64_t nitems, uint32_t ncols, uint64_t P, uint64_t W, int dtype, const Record* rec,
                              const Aux* aux, const PolyCoef* pcoef, const PolyAux* poly, uint64_t* words,
                              uint32_t* err, cudaStream_t st);
// poly: some column has a polynomial table (its tiles then get the exact polynomial bounds)
cudaError_t launch_tile_desc_multi(const ColumnView* views, const uint64_t* tile_base, uint32_t ncols, uint64_t T,
                                   bool poly, TileDesc* tiles, cudaStream_t st);

// largest c < ncols with base[c] <= x (base nondecreasing, base[ncols] > x)
__device__ __forceinline__ uint32_t find_col(const uint64_t* __restrict__ base, uint32_t ncols, uint64_t x) {
  uint32_t lo = 0, hi = ncols;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Shape of the batched encode: values per pack item (a run of short partitions staged by one copy:
// 1024, 2048 or 4096) and fit CTAs per SM (2, 3 or 4; fewer keep more of each partition in L2 for
// the fit's second pass). Tuned per value width by leco_tune_batch_encode.
struct EncodeConfig {
  uint32_t item_values;
  uint32_t fit_ctas;
};
EncodeConfig encode_config_lookup(int dtype);
void encode_config_store(int dtype, EncodeConfig cfg);

// tuning table (tune.cu): op 0 = decode, 1 = filter-sum; keyed by value width and widest partition
ScanConfig scan_config_for(const ColumnView& c, int op);
ScanConfig scan_config_lookup(int op, int dtype, uint32_t stage_bytes);
void scan_config_store(int op, int dtype, uint32_t stage_bytes, ScanConfig cfg);

// encode pipeline (k_encode.cu). pcoef / poly: per-partition polynomial blocks (written by the fit
// of a LECO_MODEL_POLY column, read by the decode-table build and the packer) and the derived
// polynomial decode table; both nullptr for constant and linear columns.
cudaError_t launch_fit(const void* values, int dtype, uint64_t n, const uint64_t* starts,
                       uint32_t L, uint64_t m, int model, Record* rec, uint64_t* lenbits, PolyCoef* pcoef,
                       uint32_t* max_b, uint32_t* err, cudaStream_t st);
cudaError_t launch_offsets(Record* rec, const uint64_t* lenbits, uint64_t m, uint64_t* scratch,
                           uint64_t scratch_elems, uint64_t* total_out, cudaStream_t st);
uint64_t offsets_scratch_elems(uint64_t m);
cudaError_t launch_build_aux(const Record* rec, const PolyCoef* pcoef, uint64_t m, uint64_t n, Aux* aux,
                             PolyAux* poly, uint32_t* status, cudaStream_t st);
cudaError_t launch_pack(const void* values, int dtype, const Record* rec, const Aux* aux, const PolyCoef* pcoef,
                        const PolyAux* poly, uint64_t m, uint64_t n, uint64_t total_bits, uint64_t* words,
                        uint64_t nwords, uint32_t* err, cudaStream_t st);
// the same for a column of constant and linear partitions of any lengths (variable partitions):
// short partitions that start in one 2048-position window share one staged copy
cudaError_t launch_pack_var(const void* values, int dtype, const Record* rec, const Aux* aux, uint64_t m, uint64_t n,
                            uint64_t total_bits, uint64_t* words, uint64_t nwords, uint32_t* err, cudaStream_t st);

// scans (k_scan.cu) and lookups (k_decode.cu)
cudaError_t launch_tile_desc(const ColumnView& c, TileDesc* tiles, cudaStream_t st);
cudaError_t launch_wait_selftest(uint64_t limit_ns, uint32_t* status, cudaStream_t st);
cudaError_t launch_decode(const ColumnView& c, uint64_t begin, uint64_t count, void* out,
                          cudaStream_t st);
cudaError_t launch_filter_sum(const ColumnView& c, uint64_t lo, uint64_t hi, uint32_t flags,
                              leco_sum_result* out, cudaStream_t st);
cudaError_t launch_filter_sum_cfg(const ColumnView& c, uint64_t lo, uint64_t hi, uint32_t flags,
                                  leco_sum_result* out, ScanConfig cfg, cudaStream_t st);
cudaError_t launch_decode_cfg(const ColumnView& c, uint64_t begin, uint64_t count, void* out,
                              ScanConfig cfg, cudaStream_t st);
cudaError_t launch_lookup_multi(const ColumnView* views, const uint32_t* col, const uint64_t* idx, uint64_t k,
                                uint64_t* out, cudaStream_t st);
// poly: some column of the batch may hold polynomial partitions (a column with a polynomial table)
cudaError_t launch_batch_decode(const ColumnView* d_cols, const BatchItem* d_items, uint64_t nitems,
                                uint32_t stage_bytes, ScanConfig cfg, bool poly, uint32_t* status, cudaStream_t st);
cudaError_t launch_random_access(const ColumnView& c, const uint64_t* idx, uint64_t k, void* out,
                                 cudaStream_t st);

// variable partitioner (k_var.cu)
cudaError_t search_partition_size(const void* values, int dtype, uint64_t n, int model, uint32_t N, double frac,
                                  uint64_t seed, uint32_t* best_L, uint64_t* best_bits, uint64_t* evals,
                                  cudaStream_t st);
cudaError_t var_partition(const void* values, int dtype, uint64_t n, double tau, uint32_t cap,
                          int model, uint64_t* starts_out, uint64_t* m_out, cudaStream_t st);

int sm_count();
// Stream-ordered device allocation from the library's own memory pool on the current device. The
// pool keeps freed memory for reuse (no release threshold), so repeated encodes do not map and
// unmap pages at every synchronization; leco_trim_memory hands the cached memory back.
cudaError_t dev_alloc(void** p, uint64_t bytes, cudaStream_t st);

}  // namespace leco
