// Encoder kernels (§3.1 Regressor, §3.3 Encoder): per-partition fit (fit.cuh), offset scan,
// decode-table build and residual packing.
#include "fit.cuh"
#include "leco_internal.cuh"

namespace leco {

namespace {

constexpr int kFitBlock = 256;

__device__ __forceinline__ uint64_t part_begin(const uint64_t* starts, uint32_t L, uint64_t n,
                                               uint64_t p) {
  if (starts) return starts[p];
  const uint64_t s = p * (uint64_t)L;
  return s < n ? s : n;
}

// one CTA per partition (grid-stride)
__global__ void __launch_bounds__(kFitBlock)
    k_fit(const void* __restrict__ values, int dtype, uint64_t n, const uint64_t* __restrict__ starts,
          uint32_t L, uint64_t m, int model, Record* __restrict__ rec, uint64_t* __restrict__ lenbits,
          uint32_t* __restrict__ max_b) {
  __shared__ FitShared sm;
  for (uint64_t p = blockIdx.x; p < m; p += gridDim.x) {
    const uint64_t a = part_begin(starts, L, n, p);
    const uint64_t e = part_begin(starts, L, n, p + 1);
    const uint32_t N = (uint32_t)(e - a);
    const FitResult R = fit_range<kFitBlock>(values, dtype, a, N, model, threadIdx.x, &sm);
    if (threadIdx.x == 0) {
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

__global__ void k_build_aux(const Record* __restrict__ rec, uint64_t m, uint64_t n, Aux* __restrict__ aux) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < m;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const Record r = rec[p];
    const uint64_t e = p + 1 < m ? rec[p + 1].start : n;
    aux[p] = aux_of(r, e > r.start ? e - r.start : 0);
  }
}

// ------------------------------------------------------------------------------ packing

// Gather packing: thread per output word. The word's bits [64w, 64w+64) are filled from the
// fields that overlap it (first partition by a search over the offsets), each field recomputed
// from the input value and the partition's prediction. No atomics, no pre-zeroing.
__device__ uint64_t pack_word(const void* __restrict__ values, int dtype, const Record* __restrict__ rec,
                              const Aux* __restrict__ aux, uint64_t m, uint64_t n, uint64_t total_bits,
                              uint64_t w) {
  {
    const uint64_t bit0 = w * 64;
    if (bit0 >= total_bits) return 0;
    uint64_t lo = 0, hi = m;  // largest p with off(p) <= bit0
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) >> 1;
      if (w3_off(__ldg(&aux[mid].word3)) <= bit0)
        lo = mid;
      else
        hi = mid;
    }
    uint64_t acc = 0;
    const uint64_t end = bit0 + 64;
    for (uint64_t p = lo; p < m; p++) {
      const Aux a = aux[p];
      const uint64_t off = w3_off(a.word3);
      if (off >= end) break;
      const uint32_t b = w3_b(a.word3);
      if (b == 0) continue;
      const uint64_t pe = p + 1 < m ? aux[p + 1].start : n;
      const uint32_t N = (uint32_t)(pe - a.start);
      uint32_t x = bit0 > off ? (uint32_t)(bit0 - off) / b : 0u;  // < 2^30 bits per partition
      uint64_t fpos = off + (uint64_t)x * b;
      for (; x < N && fpos < end; x++, fpos += b) {
        const uint64_t v = load_value(values, dtype, a.start + x);
        const int64_t pred = predict_aux(a, rec, p, x);
        const uint64_t z = zz_encode((int64_t)(v - (uint64_t)pred));
        if (fpos >= bit0)
          acc |= z << (uint32_t)(fpos - bit0);
        else
          acc |= z >> (uint32_t)(bit0 - fpos);
      }
      if (x < N) break;
    }
    return acc;
  }
}

__global__ void __launch_bounds__(256)
    k_pack(const void* __restrict__ values, int dtype, const Record* __restrict__ rec,
           const Aux* __restrict__ aux, uint64_t m, uint64_t n, uint64_t total_bits,
           uint64_t* __restrict__ words, uint64_t nwords) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < nwords;
       w += (uint64_t)gridDim.x * blockDim.x)
    words[w] = pack_word(values, dtype, rec, aux, m, n, total_bits, w);
}

// ------------------------------------------------------------------------------ batched encode

// CTA per partition of every column: the partition's column by a search over part_base
__global__ void __launch_bounds__(kFitBlock)
    k_fit_multi(const EncCol* __restrict__ cols, const uint64_t* __restrict__ part_base, uint32_t ncols,
                uint64_t P, int dtype, Record* __restrict__ rec, uint64_t* __restrict__ lenbits,
                uint32_t* __restrict__ max_b) {
  __shared__ FitShared sm;
  for (uint64_t p = blockIdx.x; p < P; p += gridDim.x) {
    const uint32_t c = find_col(part_base, ncols, p);
    const EncCol col = cols[c];
    const uint64_t a = (p - part_base[c]) * (uint64_t)col.L;
    const uint64_t e = a + col.L < col.n ? a + col.L : col.n;
    const uint32_t N = (uint32_t)(e - a);
    const FitResult R = fit_range<kFitBlock>(col.values, dtype, a, N, col.model, threadIdx.x, &sm);
    if (threadIdx.x == 0) {
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
                                    uint32_t ncols, uint64_t P, uint64_t* __restrict__ col_bits) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = find_col(part_base, ncols, p);
    const uint64_t base = off[part_base[c]];
    rec[p].word3 = (rec[p].word3 & ~kOffMask) | ((off[p] - base) & kOffMask);
    if (p + 1 == part_base[c + 1]) col_bits[c] = off[p] + lenbits[p] - base;
  }
}

__global__ void k_aux_multi(const Record* __restrict__ rec, const EncCol* __restrict__ cols,
                            const uint64_t* __restrict__ part_base, uint32_t ncols, uint64_t P,
                            Aux* __restrict__ aux) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < P;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = find_col(part_base, ncols, p);
    const Record r = rec[p];
    const uint64_t e = p + 1 < part_base[c + 1] ? rec[p + 1].start : cols[c].n;
    aux[p] = aux_of(r, e > r.start ? e - r.start : 0);
  }
}

__global__ void __launch_bounds__(256)
    k_pack_multi(const EncCol* __restrict__ cols, const uint64_t* __restrict__ part_base,
                 const uint64_t* __restrict__ word_base, const uint64_t* __restrict__ col_bits, uint32_t ncols,
                 uint64_t W, int dtype, const Record* __restrict__ rec, const Aux* __restrict__ aux,
                 uint64_t* __restrict__ words) {
  for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < W;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = find_col(word_base, ncols, w);
    const uint64_t p0 = part_base[c];
    words[w] = pack_word(cols[c].values, dtype, rec + p0, aux + p0, part_base[c + 1] - p0, cols[c].n, col_bits[c],
                         w - word_base[c]);
  }
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

cudaError_t launch_fit(const void* values, int dtype, uint64_t n, const uint64_t* starts,
                       uint32_t L, uint64_t m, int model, Record* rec, uint64_t* lenbits,
                       uint32_t* max_b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(max_b, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess || m == 0) return e;
  const uint64_t cap = (uint64_t)sm_count() * 16;
  const int grid = (int)(m < cap ? m : cap);
  k_fit<<<grid, kFitBlock, 0, st>>>(values, dtype, n, starts, L, m, model, rec, lenbits, max_b);
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

cudaError_t launch_build_aux(const Record* rec, uint64_t m, uint64_t n, Aux* aux, uint32_t* status,
                             cudaStream_t st) {
  (void)status;
  if (m == 0) return cudaSuccess;
  k_build_aux<<<grid_for(m, 256, 8), 256, 0, st>>>(rec, m, n, aux);
  return cudaGetLastError();
}

cudaError_t launch_pack(const void* values, int dtype, const Record* rec, const Aux* aux,
                        uint64_t m, uint64_t n, uint64_t total_bits, uint64_t* words,
                        uint64_t nwords, cudaStream_t st) {
  if (nwords == 0) return cudaSuccess;
  k_pack<<<grid_for(nwords, 256, 8), 256, 0, st>>>(values, dtype, rec, aux, m, n, total_bits, words,
                                                   nwords);
  return cudaGetLastError();
}

cudaError_t launch_fit_multi(const EncCol* cols, const uint64_t* part_base, uint32_t ncols, uint64_t P, int dtype,
                             Record* rec, uint64_t* lenbits, uint32_t* max_b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(max_b, 0, sizeof(uint32_t) * (ncols ? ncols : 1), st);
  if (e != cudaSuccess || P == 0) return e;
  const uint64_t cap = (uint64_t)sm_count() * 16;
  k_fit_multi<<<(int)(P < cap ? P : cap), kFitBlock, 0, st>>>(cols, part_base, ncols, P, dtype, rec, lenbits, max_b);
  return cudaGetLastError();
}

uint64_t offsets_multi_scratch_elems(uint64_t P) { return P + (P + kPrefixTile - 1) / kPrefixTile + 2; }

cudaError_t launch_offsets_multi(Record* rec, const uint64_t* lenbits, const uint64_t* part_base, uint32_t ncols,
                                 uint64_t P, uint64_t* scratch, uint64_t* col_bits, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(col_bits, 0, sizeof(uint64_t) * (ncols ? ncols : 1), st);
  if (e != cudaSuccess || P == 0) return e;
  uint64_t* off = scratch;
  uint64_t* tiles = scratch + P;
  uint64_t* total = scratch + offsets_multi_scratch_elems(P) - 1;
  e = scan_u64(lenbits, P, off, tiles, total, st);
  if (e != cudaSuccess) return e;
  k_set_offsets_multi<<<grid_for(P, 256, 8), 256, 0, st>>>(rec, off, lenbits, part_base, ncols, P, col_bits);
  return cudaGetLastError();
}

cudaError_t launch_aux_multi(const Record* rec, const EncCol* cols, const uint64_t* part_base, uint32_t ncols,
                             uint64_t P, Aux* aux, cudaStream_t st) {
  if (P == 0) return cudaSuccess;
  k_aux_multi<<<grid_for(P, 256, 8), 256, 0, st>>>(rec, cols, part_base, ncols, P, aux);
  return cudaGetLastError();
}

cudaError_t launch_pack_multi(const EncCol* cols, const uint64_t* part_base, const uint64_t* word_base,
                              const uint64_t* col_bits, uint32_t ncols, uint64_t W, int dtype, const Record* rec,
                              const Aux* aux, uint64_t* words, cudaStream_t st) {
  if (W == 0) return cudaSuccess;
  k_pack_multi<<<grid_for(W, 256, 8), 256, 0, st>>>(cols, part_base, word_base, col_bits, ncols, W, dtype, rec, aux,
                                                    words);
  return cudaGetLastError();
}

}  // namespace leco
