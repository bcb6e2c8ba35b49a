// assemble.cu -- tally assembly: detection events (v, j) -> the count matrix
// C_jv of Eq. (IMC) (Sec. 5.1: T_ij estimated by Monte Carlo; Sec. 2: tallies
// are counts of histories).
//
// Events arrive as 64-bit keys v*M + j in arbitrary order (the transport
// kernel appends them with atomics).  A stable LSD radix sort orders them by
// (v, j); a run-length pass turns runs of equal keys into (v, j, count)
// triples, which are the CSC form.  The CSR form comes from a second radix
// sort of the (j*N + v, count) pairs.  Everything is integer work, so the
// matrix is bit-identical from run to run.  No floating-point atomics.
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <vector>

#include "internal.cuh"

namespace mcs {

// ---------------------------------------------------------------------------
// exclusive scan (u32), reduce-then-scan over tiles of 2048 elements
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;  // inclusive per warp
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  const uint32_t before = warp > 0 ? s_warp[warp - 1] : 0u;
  return before + x - v;
}

__global__ void scan_reduce_kernel(const uint32_t *in, uint32_t *sums, int64_t n) {
  __shared__ uint32_t s_warp[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  uint32_t total;
  block_exclusive_scan(acc, s_warp, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_apply_kernel(const uint32_t *in, uint32_t *out, const uint32_t *offsets, int64_t n) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_items[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  // coalesced load into shared memory, then each thread scans 8 consecutive items
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    s_items[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0u;
  }
  __syncthreads();
  uint32_t local[kScanItems];
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    local[k] = acc;
    acc += s_items[threadIdx.x * kScanItems + k];
  }
  uint32_t total;
  const uint32_t pre = block_exclusive_scan(acc, s_warp, total) + (offsets ? offsets[blockIdx.x] : 0u);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s_items[threadIdx.x * kScanItems + k] = pre + local[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) out[i] = s_items[k * kScanThreads + threadIdx.x];
  }
}

int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s) {
  if (n <= 0) return MC_OK;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    count_launch(); scan_apply_kernel<<<1, kScanThreads, 0, s>>>(in, out, nullptr, n);
    MCS_LAUNCHED();
    return MC_OK;
  }
  DevBuf sums, offs;
  MCS_TRY(sums.alloc(tiles * sizeof(uint32_t), s));
  MCS_TRY(offs.alloc(tiles * sizeof(uint32_t), s));
  count_launch(); scan_reduce_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, sums.as<uint32_t>(), n);
  MCS_LAUNCHED();
  MCS_TRY(exclusive_scan_u32(sums.as<uint32_t>(), offs.as<uint32_t>(), tiles, s));
  count_launch(); scan_apply_kernel<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, offs.as<uint32_t>(), n);
  MCS_LAUNCHED();
  return MC_OK;
}

// ---------------------------------------------------------------------------
// LSD radix sort of u64 keys (optional u32 payload), 8-bit digits
// ---------------------------------------------------------------------------
// Per pass: a histogram of the digit per tile of kSortTile keys, an exclusive
// scan of the digit-major counts (global start of each (digit, tile)), and a
// stable scatter.  The scatter first orders the tile by digit in shared
// memory, then writes the tile out in that order, so that each digit's run
// goes to consecutive addresses.  Within the tile, warp w holds the
// contiguous positions [w * 32 * kSortRounds, (w + 1) * 32 * kSortRounds):
// each warp ranks its keys among its own keys of the same digit (running
// per-warp digit counters), and a key's place in the ordered tile is the
// digit's start in the tile, plus the keys of that digit in earlier warps,
// plus its rank -- the tile order, so the sort is stable.
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 12;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 3072 keys

__global__ void radix_hist_kernel(const uint64_t *keys, int64_t n, int shift, uint32_t *counts, int64_t n_tiles) {
  __shared__ uint32_t s_hist[256];
  s_hist[threadIdx.x] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&s_hist[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * n_tiles + blockIdx.x] = s_hist[threadIdx.x];
}

// exclusive scan of one value per thread over a 256-thread block
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t *s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  return before + x - v;
}

// Stable scatter: the key at tile position p goes to
//   offset[digit][tile] + (number of earlier keys of this tile with the same digit).
template <bool VALS>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(const uint64_t *kin, const uint32_t *vin,
                                                                     uint64_t *kout, uint32_t *vout, int64_t n,
                                                                     int shift, const uint32_t *counts,
                                                                     const uint32_t *offsets, int64_t n_tiles) {
  constexpr int kWarps = kSortThreads / 32;
  constexpr int kWarpKeys = 32 * kSortRounds;
  constexpr uint32_t kNone = 0xFFFFFFFFu;
  __shared__ uint64_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[VALS ? kSortTile : 1];
  __shared__ uint32_t s_shift[256], s_start[256], s_warp[kWarps];
  __shared__ uint32_t s_wc[kWarps][256];  // per warp and digit: keys so far, then the warp's start in the tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t tile_off = (int64_t)threadIdx.x * n_tiles + blockIdx.x;
  const uint32_t start = block_exclusive_scan_256(counts[tile_off], s_warp);
  s_start[threadIdx.x] = start;
  // output position of ordered-tile position p with this digit: p + shift
  // (the digit's global start minus its start in the tile, modulo 2^32)
  s_shift[threadIdx.x] = offsets[tile_off] - start;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s_wc[w][threadIdx.x] = 0u;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  const int64_t left = n - base;
  const int cnt = left < kSortTile ? (int)left : kSortTile;
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t *wc = s_wc[warp];
  uint64_t key[kSortRounds];
  uint32_t val[kSortRounds];
  uint32_t slot[kSortRounds];  // digit | (rank among the warp's keys of that digit) << 8
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int p = warp * kWarpKeys + r * 32 + lane;
    key[r] = p < cnt ? kin[base + p] : 0ull;
    if (VALS) val[r] = p < cnt ? vin[base + p] : 0u;
  }
  // 1. rank each key among the warp's keys of its digit, in tile order
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const bool valid = warp * kWarpKeys + r * 32 + lane < cnt;
    const uint32_t digit = valid ? (uint32_t)((key[r] >> shift) & 255u) : 256u;
    // lanes holding the same digit: one vote per digit bit (and one on
    // validity), intersected -- measured faster in this kernel than
    // match.any (the same masks)
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    if (!valid) peers = ~peers;
#pragma unroll
    for (int bit = 0; bit < 8; ++bit) {
      const uint32_t bb = __ballot_sync(0xffffffffu, (digit >> bit) & 1u);
      peers &= ((digit >> bit) & 1u) ? bb : ~bb;
    }
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0u;
    if (valid && lane == leader) before = wc[digit];
    before = __shfl_sync(0xffffffffu, before, leader);
    if (valid && lane == leader) wc[digit] = before + __popc(peers);
    __syncwarp();
    slot[r] = valid ? digit | ((before + __popc(peers & lt_mask)) << 8) : kNone;
  }
  __syncthreads();
  // 2. per digit: each warp's start in the ordered tile
  {
    uint32_t run = s_start[threadIdx.x];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = s_wc[w][threadIdx.x];
      s_wc[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
  // 3. order the tile by digit in shared memory
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    if (slot[r] != kNone) {
      const uint32_t pos = wc[slot[r] & 255u] + (slot[r] >> 8);
      s_keys[pos] = key[r];
      if (VALS) s_vals[pos] = val[r];
    }
  }
  __syncthreads();
  // 4. write the tile out in digit order: each digit's keys are consecutive
  for (int p = threadIdx.x; p < cnt; p += kSortThreads) {
    const uint64_t k = s_keys[p];
    const uint32_t pos = (uint32_t)p + s_shift[(uint32_t)((k >> shift) & 255u)];
    kout[pos] = k;
    if (VALS) vout[pos] = s_vals[p];
  }
}

int radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int bits,
                   bool *result_in_alt, cudaStream_t s, int first_bit) {
  *result_in_alt = false;
  if (n <= 1 || bits <= 0) return MC_OK;
  if (n >= (int64_t)0xFFFFFFFFll) {
    set_error("radix sort: %lld keys exceed the 32-bit offset range", (long long)n);
    return MC_EINVAL;
  }
  const int64_t n_tiles = (n + kSortTile - 1) / kSortTile;
  DevBuf counts, offsets;
  MCS_TRY(counts.alloc(256 * n_tiles * sizeof(uint32_t), s));
  MCS_TRY(offsets.alloc(256 * n_tiles * sizeof(uint32_t), s));
  uint64_t *kin = keys, *kout = keys_alt;
  uint32_t *vin = vals, *vout = vals_alt;
  bool in_alt = false;
  for (int shift = first_bit; shift < bits; shift += 8) {
    count_launch(); radix_hist_kernel<<<(unsigned)n_tiles, kSortThreads, 0, s>>>(kin, n, shift, counts.as<uint32_t>(), n_tiles);
    MCS_LAUNCHED();
    MCS_TRY(exclusive_scan_u32(counts.as<uint32_t>(), offsets.as<uint32_t>(), 256 * n_tiles, s));
    count_launch();
    if (vin)
      radix_scatter_kernel<true><<<(unsigned)n_tiles, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift,
                                                                           counts.as<uint32_t>(),
                                                                           offsets.as<uint32_t>(), n_tiles);
    else
      radix_scatter_kernel<false><<<(unsigned)n_tiles, kSortThreads, 0, s>>>(kin, nullptr, kout, nullptr, n, shift,
                                                                            counts.as<uint32_t>(),
                                                                            offsets.as<uint32_t>(), n_tiles);
    MCS_LAUNCHED();
    uint64_t *tk = kin; kin = kout; kout = tk;
    uint32_t *tv = vin; vin = vout; vout = tv;
    in_alt = !in_alt;
  }
  *result_in_alt = in_alt;
  return MC_OK;
}

// ---------------------------------------------------------------------------
// run-length encoding of sorted keys
// ---------------------------------------------------------------------------
__global__ void head_flags_kernel(const uint64_t *keys, int64_t n, uint32_t *flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void compact_heads_kernel(const uint64_t *keys, const uint32_t *flags, const uint32_t *idx, int64_t n,
                                     uint64_t *ukeys, uint32_t *upos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (flags[i]) {
      ukeys[idx[i]] = keys[i];
      upos[idx[i]] = (uint32_t)i;
    }
  }
}

__global__ void run_lengths_kernel(const uint32_t *upos, int64_t nu, int64_t n, uint32_t *cnt) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x)
    cnt[u] = (u + 1 < nu ? upos[u + 1] : (uint32_t)n) - upos[u];
}

// (v*M + j) -> row j, column v; histogram of the column (or row) index.
__global__ void split_keys_kernel(const uint64_t *ukeys, int64_t nu, uint64_t m, uint32_t *major_out,
                                  uint32_t *minor_out, uint32_t *major_hist) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = ukeys[u];
    const uint32_t major = (uint32_t)(k / m), minor = (uint32_t)(k % m);
    if (major_out) major_out[u] = major;
    minor_out[u] = minor;
    atomicAdd(&major_hist[major], 1u);
  }
}

// Pointer array of a sorted sequence of major indices: ptr[c] = the first
// position whose major index is >= c, ptr[n_major] = nu.  Position u writes
// the entries c in (major of u - 1, major of u] (the last position also
// (major, n_major]), so every entry is written once and no histogram or scan
// is needed.
__device__ __forceinline__ void fill_ptr(uint32_t *ptr, int64_t u, int64_t nu, int64_t major, int64_t prev,
                                         int64_t n_major) {
  for (int64_t c = prev + 1; c <= major; ++c) ptr[c] = (uint32_t)u;
  if (u == nu - 1)
    for (int64_t c = major + 1; c <= n_major; ++c) ptr[c] = (uint32_t)nu;
}

// Sorted unique keys v*M + j -> CSC row indices j, col_ptr, and the
// transposed keys (j << b) | v for the CSR.  The loop runs the same number of
// times on every thread of a block (the shuffle needs whole warps).
__global__ void csc_split_kernel(const uint64_t *ukeys, int64_t nu, uint64_t m, int b, uint32_t *row_idx,
                                 uint32_t *col_ptr, int64_t n_cols, uint64_t *tkeys) {
  const int lane = threadIdx.x & 31;
  for (int64_t u0 = (int64_t)blockIdx.x * blockDim.x; u0 < nu; u0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = u0 + threadIdx.x;
    const bool valid = u < nu;
    const uint64_t k = valid ? ukeys[u] : 0ull;
    const uint64_t v = k / m, j = k - v * m;
    uint64_t vp = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 0) vp = (valid && u > 0) ? ukeys[u - 1] / m : 0ull;
    if (valid) {
      row_idx[u] = (uint32_t)j;
      tkeys[u] = (j << b) | v;
      fill_ptr(col_ptr, u, nu, (int64_t)v, u == 0 ? -1 : (int64_t)vp, n_cols);
    }
  }
}

// Sorted keys (j << b) | v -> CSR column indices v and row_ptr.
__global__ void csr_split_kernel(const uint64_t *tkeys, int64_t nu, int b, uint32_t *col_idx, uint32_t *row_ptr,
                                 int64_t n_rows) {
  const uint64_t mask = (1ull << b) - 1ull;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = tkeys[u];
    col_idx[u] = (uint32_t)(k & mask);
    fill_ptr(row_ptr, u, nu, (int64_t)(k >> b), u == 0 ? -1 : (int64_t)(tkeys[u - 1] >> b), n_rows);
  }
}

// n_v = #{h in [first, first+count) : h mod N = v}
__global__ void histories_per_voxel_kernel(uint64_t first, uint64_t count, uint64_t n_vox, uint32_t *n_v,
                                           float *inv_n) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vox; v += (uint64_t)gridDim.x * blockDim.x) {
    // number of h in [0, x) with h = v (mod N)
    auto below = [&](uint64_t x) -> uint64_t { return x > v ? (x - v - 1) / n_vox + 1 : 0; };
    const uint64_t c = below(first + count) - below(first);
    n_v[v] = (uint32_t)c;
    inv_n[v] = c ? (float)(1.0 / (double)c) : 0.0f;
  }
}

// S_v = sum_j C_jv over CSC column v, and the largest count.
__global__ void column_sums_kernel(const uint32_t *col_ptr, const uint32_t *cnt, int64_t n_cols, double *colsum,
                                   float *inv_colsum, unsigned int *max_count) {
  uint32_t mymax = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_cols; v += (int64_t)gridDim.x * blockDim.x) {
    uint64_t acc = 0;
    for (uint32_t k = col_ptr[v]; k < col_ptr[v + 1]; ++k) {
      acc += cnt[k];
      mymax = cnt[k] > mymax ? cnt[k] : mymax;
    }
    colsum[v] = (double)acc;
    inv_colsum[v] = acc ? (float)(1.0 / (double)acc) : 0.0f;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, mymax, o);
    mymax = y > mymax ? y : mymax;
  }
  if ((threadIdx.x & 31) == 0 && mymax) atomicMax(max_count, mymax);
}

// Weighted tallies (forced detection): the weight sum of each run of equal
// keys, wsum[u] = sum of w[perm[e]] over the run's sorted positions e, as an
// exact 64-bit integer sum (the weights are fixed point).
__global__ void iota_kernel(uint32_t *out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (uint32_t)i;
}

// A CSC entry's weight sum and count side by side, so that the CSR can
// gather both with one 16-byte load.
struct alignas(16) WEntry {
  uint64_t w;
  uint32_t cnt, pad;
};

__global__ void run_weights_kernel(const uint32_t *upos, const uint32_t *ucnt, int64_t nu, const uint32_t *perm,
                                   const uint64_t *w, uint64_t *wsum, WEntry *ent) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += (int64_t)gridDim.x * blockDim.x) {
    uint64_t acc = 0;
    const uint32_t c = ucnt[u], b = upos[u], e = b + c;
    for (uint32_t k = b; k < e; ++k) acc += w[perm[k]];
    wsum[u] = acc;
    WEntry x;
    x.w = acc; x.cnt = c; x.pad = 0u;
    ent[u] = x;
  }
}

// out_cnt[i] = ent[perm[i]].cnt, out_w[i] = ent[perm[i]].w
__global__ void gather_entries_kernel(const uint32_t *perm, int64_t n, const WEntry *ent, uint32_t *out_cnt,
                                      uint64_t *out_w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const WEntry x = ent[perm[i]];
    out_cnt[i] = x.cnt;
    out_w[i] = x.w;
  }
}

// S_v = sum over column v of the fixed-point weights, in column order
__global__ void column_weight_sums_kernel(const uint32_t *col_ptr, const uint64_t *wq, int64_t n_cols, double *colsum,
                                          float *inv_colsum) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_cols; v += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (uint32_t k = col_ptr[v]; k < col_ptr[v + 1]; ++k) acc += (double)wq[k] * (1.0 / kFdScale);
    colsum[v] = acc;
    inv_colsum[v] = acc > 0.0 ? (float)(1.0 / acc) : 0.0f;
  }
}

static int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)device_sm_count() * 32;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

static int bits_for(uint64_t range) {
  int b = 0;
  while (b < 64 && (range >> b) != 0) ++b;
  return b;
}

// ---------------------------------------------------------------------------
// assembly by buckets (unweighted events, short columns and rows)
// ---------------------------------------------------------------------------
// Events are counted per column and each event's row is placed in its
// column's bucket (in any order); every bucket is then sorted by row, one
// thread per bucket, with equal rows merged into a count.  The CSR is made
// the same way from the CSC entries.  Sorting makes the result unique: the
// same sorted, merged CSC and CSR as the radix path, in a few passes over
// the events instead of one per digit.  Taken only when no column holds more
// than kBucketLen events and no row more than kBucketLen entries.
constexpr int kBucketLen = 64;

__global__ void bucket_count_kernel(const uint64_t *keys, int64_t n, uint64_t m, uint32_t *cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[keys[i] / m], 1u);
}

// event i -> its row, at start[column] + (its place among the column's
// events, in arrival order at the atomic)
__global__ void bucket_fill_kernel(const uint64_t *keys, int64_t n, uint64_t m, const uint32_t *start,
                                   uint32_t *cursor, uint32_t *minor) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const uint64_t v = k / m;
    minor[start[v] + atomicAdd(&cursor[v], 1u)] = (uint32_t)(k - v * m);
  }
}

// Compare-exchange of (a[i], w[i]) and (a[k], w[k]) by a.
__device__ __forceinline__ void cmp_swap(uint32_t &ai, uint32_t &wi, uint32_t &ak, uint32_t &wk) {
  if (ak < ai) {
    const uint32_t t = ai, u = wi;
    ai = ak; wi = wk;
    ak = t; wk = u;
  }
}

// Sort bucket c = [start[c], start[c + 1]) of `minor` ascending, with its
// payload (cnt_in, or 1 per element when cnt_in is NULL), merge equal
// values (payloads summed) and write the u merged values and payloads to
// the bucket's first u places of minor and cnt_out; uniq[c] = u.  Buckets of
// up to 8 elements are sorted in registers (Batcher's odd-even merge
// network, unused places holding the largest value); longer ones, up to
// kBucketLen, by insertion in a local array.  A longer bucket sets
// *overflow and is left as it is.
__global__ void bucket_sort_merge_kernel(const uint32_t *start, int64_t n_major, uint32_t *minor,
                                         const uint32_t *cnt_in, uint32_t *cnt_out, uint32_t *uniq,
                                         unsigned int *overflow) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_major;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = start[c];
    const int len = (int)(start[c + 1] - b);
    if (len > kBucketLen) {
      atomicOr(overflow, 1u);
      continue;
    }
    if (len <= 8) {
      uint32_t r[8], q[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        r[k] = k < len ? minor[b + k] : 0xffffffffu;
        q[k] = k < len ? (cnt_in ? cnt_in[b + k] : 1u) : 0u;
      }
      // odd-even merge sort of 8: sorted pairs, fours, then eight
#pragma unroll
      for (int k = 0; k < 8; k += 2) cmp_swap(r[k], q[k], r[k + 1], q[k + 1]);
#pragma unroll
      for (int k = 0; k < 8; k += 4) {
        cmp_swap(r[k], q[k], r[k + 2], q[k + 2]);
        cmp_swap(r[k + 1], q[k + 1], r[k + 3], q[k + 3]);
        cmp_swap(r[k + 1], q[k + 1], r[k + 2], q[k + 2]);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) cmp_swap(r[k], q[k], r[k + 4], q[k + 4]);
      cmp_swap(r[2], q[2], r[4], q[4]);
      cmp_swap(r[3], q[3], r[5], q[5]);
      cmp_swap(r[1], q[1], r[2], q[2]);
      cmp_swap(r[3], q[3], r[4], q[4]);
      cmp_swap(r[5], q[5], r[6], q[6]);
      // merge equal values and write, all from registers (the loads are done)
      int u = 0;
      uint32_t last = 0u, acc = 0u;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k < len) {
          if (u > 0 && r[k] == last) {
            acc += q[k];
          } else {
            if (u > 0) {
              minor[b + u - 1] = last;
              cnt_out[b + u - 1] = acc;
            }
            last = r[k];
            acc = q[k];
            ++u;
          }
        }
      }
      if (u > 0) {
        minor[b + u - 1] = last;
        cnt_out[b + u - 1] = acc;
      }
      uniq[c] = (uint32_t)u;
      continue;
    }
    uint32_t a[kBucketLen], w[kBucketLen];
    {
      for (int k = 0; k < len; ++k) {  // insertion sort while loading
        const uint32_t x = minor[b + k], y = cnt_in ? cnt_in[b + k] : 1u;
        int t = k;
        for (; t > 0 && a[t - 1] > x; --t) {
          a[t] = a[t - 1];
          w[t] = w[t - 1];
        }
        a[t] = x;
        w[t] = y;
      }
    }
    int u = 0;
    for (int k = 0; k < len; ++k) {
      if (u > 0 && a[k] == a[u - 1]) {
        w[u - 1] += w[k];
      } else {
        a[u] = a[k];
        w[u] = w[k];
        ++u;
      }
    }
    for (int k = 0; k < u; ++k) {
      minor[b + k] = a[k];
      cnt_out[b + k] = w[k];
    }
    uniq[c] = (uint32_t)u;
  }
}

// CSC: bucket c's merged entries to [col_ptr[c], col_ptr[c + 1]), and the
// number of entries of each row
__global__ void bucket_compact_kernel(const uint32_t *start, const uint32_t *col_ptr, int64_t n_cols,
                                      const uint32_t *minor, const uint32_t *cnt, uint32_t *row_idx,
                                      uint32_t *csc_cnt, uint32_t *row_hist) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cols;
       c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t b = start[c], o = col_ptr[c], u = col_ptr[c + 1] - o;
    for (uint32_t k = 0; k < u; ++k) {
      const uint32_t j = minor[b + k];
      row_idx[o + k] = j;
      csc_cnt[o + k] = cnt[b + k];
      atomicAdd(&row_hist[j], 1u);
    }
  }
}

// CSR buckets: every CSC entry (j, v) to row j's bucket (any order)
__global__ void transpose_fill_kernel(const uint32_t *col_ptr, int64_t n_cols, const uint32_t *row_idx,
                                      const uint32_t *csc_cnt, const uint32_t *row_ptr, uint32_t *cursor,
                                      uint32_t *col_idx, uint32_t *csr_cnt) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cols;
       c += (int64_t)gridDim.x * blockDim.x) {
    for (uint32_t k = col_ptr[c]; k < col_ptr[c + 1]; ++k) {
      const uint32_t j = row_idx[k];
      const uint32_t pos = row_ptr[j] + atomicAdd(&cursor[j], 1u);
      col_idx[pos] = (uint32_t)c;
      csr_cnt[pos] = csc_cnt[k];
    }
  }
}

// The CSC and CSR of n > 0 unweighted events by buckets.  Sets *done, or
// leaves the system's matrix unfinished (and the keys untouched) when a
// column or a row is too long for a bucket.
static int assemble_buckets(mc_system *sys, const uint64_t *keys, int64_t n, cudaStream_t s, bool *done) {
  *done = false;
  const int64_t M = sys->n_rows, N = sys->n_cols;
  DevBuf ccnt, start, flag;
  MCS_TRY(ccnt.alloc((size_t)(N + 1) * sizeof(uint32_t), s));
  MCS_TRY(start.alloc((size_t)(N + 1) * sizeof(uint32_t), s));
  MCS_TRY(flag.alloc(sizeof(unsigned int), s));
  MCS_CUDA(cudaMemsetAsync(ccnt.p, 0, (size_t)(N + 1) * sizeof(uint32_t), s));
  MCS_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(unsigned int), s));
  count_launch(); bucket_count_kernel<<<grid_for(n), 256, 0, s>>>(keys, n, (uint64_t)M, ccnt.as<uint32_t>());
  MCS_LAUNCHED();
  MCS_TRY(exclusive_scan_u32(ccnt.as<uint32_t>(), start.as<uint32_t>(), N + 1, s));
  // events into column buckets, sorted and merged
  DevBuf minor, ecnt;
  MCS_TRY(minor.alloc((size_t)n * sizeof(uint32_t), s));
  MCS_TRY(ecnt.alloc((size_t)n * sizeof(uint32_t), s));
  MCS_CUDA(cudaMemsetAsync(ccnt.p, 0, (size_t)(N + 1) * sizeof(uint32_t), s));  // now the bucket cursors
  count_launch();
  bucket_fill_kernel<<<grid_for(n), 256, 0, s>>>(keys, n, (uint64_t)M, start.as<uint32_t>(), ccnt.as<uint32_t>(),
                                                 minor.as<uint32_t>());
  MCS_LAUNCHED();
  // ccnt becomes the merged entries per column (ccnt[N] stays 0 for the scan)
  count_launch();
  bucket_sort_merge_kernel<<<grid_for(N), 256, 0, s>>>(start.as<uint32_t>(), N, minor.as<uint32_t>(), nullptr,
                                                       ecnt.as<uint32_t>(), ccnt.as<uint32_t>(),
                                                       flag.as<unsigned int>());
  MCS_LAUNCHED();
  MCS_TRY(sys->col_ptr.alloc((size_t)(N + 1) * sizeof(uint32_t), s));
  MCS_TRY(exclusive_scan_u32(ccnt.as<uint32_t>(), sys->col_ptr.as<uint32_t>(), N + 1, s));
  uint32_t nnz = 0, too_long = 0;
  MCS_CUDA(cudaMemcpyAsync(&nnz, sys->col_ptr.as<uint32_t>() + N, sizeof(nnz), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaMemcpyAsync(&too_long, flag.p, sizeof(too_long), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  if (too_long) return MC_OK;  // a column of more than kBucketLen events
  const size_t nnz_b = (size_t)(nnz > 0 ? nnz : 1);
  MCS_TRY(sys->row_idx.alloc(nnz_b * sizeof(uint32_t), s));
  MCS_TRY(sys->csc_cnt.alloc(nnz_b * sizeof(uint32_t), s));
  DevBuf rhist;
  MCS_TRY(rhist.alloc((size_t)(M + 1) * sizeof(uint32_t), s));
  MCS_CUDA(cudaMemsetAsync(rhist.p, 0, (size_t)(M + 1) * sizeof(uint32_t), s));
  count_launch();
  bucket_compact_kernel<<<grid_for(N), 256, 0, s>>>(start.as<uint32_t>(), sys->col_ptr.as<uint32_t>(), N,
                                                    minor.as<uint32_t>(), ecnt.as<uint32_t>(),
                                                    sys->row_idx.as<uint32_t>(), sys->csc_cnt.as<uint32_t>(),
                                                    rhist.as<uint32_t>());
  MCS_LAUNCHED();
  minor.release();
  ecnt.release();
  start.release();
  ccnt.release();
  // CSR: the CSC entries into row buckets, each sorted by column
  MCS_TRY(sys->row_ptr.alloc((size_t)(M + 1) * sizeof(uint32_t), s));
  MCS_TRY(exclusive_scan_u32(rhist.as<uint32_t>(), sys->row_ptr.as<uint32_t>(), M + 1, s));
  MCS_TRY(sys->col_idx.alloc(nnz_b * sizeof(uint32_t), s));
  MCS_TRY(sys->csr_cnt.alloc(nnz_b * sizeof(uint32_t), s));
  MCS_CUDA(cudaMemsetAsync(rhist.p, 0, (size_t)(M + 1) * sizeof(uint32_t), s));  // the row cursors
  count_launch();
  transpose_fill_kernel<<<grid_for(N), 256, 0, s>>>(sys->col_ptr.as<uint32_t>(), N, sys->row_idx.as<uint32_t>(),
                                                    sys->csc_cnt.as<uint32_t>(), sys->row_ptr.as<uint32_t>(),
                                                    rhist.as<uint32_t>(), sys->col_idx.as<uint32_t>(),
                                                    sys->csr_cnt.as<uint32_t>());
  MCS_LAUNCHED();
  // rows hold distinct columns: the sort leaves every entry (rhist takes the
  // per-row counts, unused)
  count_launch();
  bucket_sort_merge_kernel<<<grid_for(M), 256, 0, s>>>(sys->row_ptr.as<uint32_t>(), M, sys->col_idx.as<uint32_t>(),
                                                       sys->csr_cnt.as<uint32_t>(), sys->csr_cnt.as<uint32_t>(),
                                                       rhist.as<uint32_t>(), flag.as<unsigned int>());
  MCS_LAUNCHED();
  MCS_CUDA(cudaMemcpyAsync(&too_long, flag.p, sizeof(too_long), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  if (too_long) return MC_OK;  // a row of more than kBucketLen entries
  sys->nnz = nnz;
  *done = true;
  return MC_OK;
}

// Steps 1-4 of the assembly by a radix sort of the event keys (any events,
// weighted or not).
static int assemble_radix(mc_system *sys, DevBuf &keys, int64_t n, cudaStream_t s, const uint64_t *weights) {
  const uint64_t M = (uint64_t)sys->n_rows, N = (uint64_t)sys->n_cols;
  // 1. sort events by (v, j); weighted: with the event index as payload
  DevBuf alt, perm, perm_alt, went;
  MCS_TRY(alt.alloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t), s));
  if (weights) {
    MCS_TRY(perm.alloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t), s));
    MCS_TRY(perm_alt.alloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t), s));
    if (n > 0) {
      count_launch(); iota_kernel<<<grid_for(n), 256, 0, s>>>(perm.as<uint32_t>(), n);
      MCS_LAUNCHED();
    }
  }
  bool in_alt = false;
  MCS_TRY(radix_sort_u64(keys.as<uint64_t>(), alt.as<uint64_t>(), weights ? perm.as<uint32_t>() : nullptr,
                         weights ? perm_alt.as<uint32_t>() : nullptr, n, bits_for(M * N - 1), &in_alt, s));
  const uint64_t *sorted = in_alt ? alt.as<uint64_t>() : keys.as<uint64_t>();
  const uint32_t *sorted_perm = weights ? (in_alt ? perm_alt.as<uint32_t>() : perm.as<uint32_t>()) : nullptr;

  // 2. run-length encode; weighted: the CSC weight sums, and each entry's
  // weight and count side by side for the CSR gather
  int64_t nu = 0;
  DevBuf ukeys, ucnt;
  if (n > 0) {
    DevBuf flags, idx, upos;
    MCS_TRY(flags.alloc(n * sizeof(uint32_t), s));
    MCS_TRY(idx.alloc(n * sizeof(uint32_t), s));
    count_launch(); head_flags_kernel<<<grid_for(n), 256, 0, s>>>(sorted, n, flags.as<uint32_t>());
    MCS_LAUNCHED();
    MCS_TRY(exclusive_scan_u32(flags.as<uint32_t>(), idx.as<uint32_t>(), n, s));
    uint32_t last_idx = 0, last_flag = 0;
    MCS_CUDA(cudaMemcpyAsync(&last_idx, idx.as<uint32_t>() + (n - 1), 4, cudaMemcpyDeviceToHost, s));
    MCS_CUDA(cudaMemcpyAsync(&last_flag, flags.as<uint32_t>() + (n - 1), 4, cudaMemcpyDeviceToHost, s));
    MCS_CUDA(cudaStreamSynchronize(s));
    nu = (int64_t)last_idx + last_flag;
    MCS_TRY(ukeys.alloc(nu * sizeof(uint64_t), s));
    MCS_TRY(upos.alloc(nu * sizeof(uint32_t), s));
    MCS_TRY(ucnt.alloc(nu * sizeof(uint32_t), s));
    count_launch(); compact_heads_kernel<<<grid_for(n), 256, 0, s>>>(sorted, flags.as<uint32_t>(), idx.as<uint32_t>(), n,
                                                     ukeys.as<uint64_t>(), upos.as<uint32_t>());
    MCS_LAUNCHED();
    count_launch(); run_lengths_kernel<<<grid_for(nu), 256, 0, s>>>(upos.as<uint32_t>(), nu, n, ucnt.as<uint32_t>());
    MCS_LAUNCHED();
    if (weights) {
      MCS_TRY(sys->csc_wq.alloc(nu * sizeof(uint64_t), s));
      MCS_TRY(went.alloc(nu * sizeof(WEntry), s));
      count_launch();
      run_weights_kernel<<<grid_for(nu), 256, 0, s>>>(upos.as<uint32_t>(), ucnt.as<uint32_t>(), nu, sorted_perm,
                                                      weights, sys->csc_wq.as<uint64_t>(), went.as<WEntry>());
      MCS_LAUNCHED();
    }
  }
  alt.release();
  perm.release();
  perm_alt.release();
  keys.release();
  sys->nnz = nu;

  // 3. CSC: rows, counts and col_ptr in sorted order; the transposed keys
  const size_t nnz_b = (size_t)(nu > 0 ? nu : 1);
  const int b = bits_for(N - 1);
  DevBuf tkeys;
  {
    MCS_TRY(sys->col_ptr.alloc((N + 1) * sizeof(uint32_t), s));
    MCS_TRY(sys->row_idx.alloc(nnz_b * sizeof(uint32_t), s));
    MCS_TRY(sys->csc_cnt.alloc(nnz_b * sizeof(uint32_t), s));
    if (weights && nu == 0) MCS_TRY(sys->csc_wq.alloc(sizeof(uint64_t), s));
    if (nu > 0) {
      MCS_TRY(tkeys.alloc(nu * sizeof(uint64_t), s));
      count_launch();
      csc_split_kernel<<<grid_for(nu), 256, 0, s>>>(ukeys.as<uint64_t>(), nu, M, b, sys->row_idx.as<uint32_t>(),
                                                    sys->col_ptr.as<uint32_t>(), (int64_t)N, tkeys.as<uint64_t>());
      MCS_LAUNCHED();
      MCS_CUDA(cudaMemcpyAsync(sys->csc_cnt.p, ucnt.p, nu * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    } else {
      MCS_CUDA(cudaMemsetAsync(sys->col_ptr.p, 0, (N + 1) * sizeof(uint32_t), s));
    }
  }
  ukeys.release();

  // 4. CSR: sort the transposed keys (with the counts, or, weighted, the CSC
  // position of each entry), then columns and row_ptr in sorted order
  {
    MCS_TRY(sys->row_ptr.alloc((M + 1) * sizeof(uint32_t), s));
    MCS_TRY(sys->col_idx.alloc(nnz_b * sizeof(uint32_t), s));
    MCS_TRY(sys->csr_cnt.alloc(nnz_b * sizeof(uint32_t), s));
    if (nu > 0) {
      DevBuf tkeys_alt, tcnt_alt, tperm;
      MCS_TRY(tkeys_alt.alloc(nu * sizeof(uint64_t), s));
      MCS_TRY(tcnt_alt.alloc(nu * sizeof(uint32_t), s));
      if (weights) {
        MCS_TRY(tperm.alloc(nu * sizeof(uint32_t), s));
        count_launch(); iota_kernel<<<grid_for(nu), 256, 0, s>>>(tperm.as<uint32_t>(), nu);
        MCS_LAUNCHED();
      }
      uint32_t *payload = weights ? tperm.as<uint32_t>() : ucnt.as<uint32_t>();
      bool talt = false;
      // the entries are in (v, j) order: a stable sort on the j bits of
      // (j << b) | v alone gives (j, v) order
      MCS_TRY(radix_sort_u64(tkeys.as<uint64_t>(), tkeys_alt.as<uint64_t>(), payload,
                             tcnt_alt.as<uint32_t>(), nu, b + bits_for(M - 1), &talt, s, b));
      const uint64_t *tk = talt ? tkeys_alt.as<uint64_t>() : tkeys.as<uint64_t>();
      const uint32_t *tc = talt ? tcnt_alt.as<uint32_t>() : payload;
      count_launch();
      csr_split_kernel<<<grid_for(nu), 256, 0, s>>>(tk, nu, b, sys->col_idx.as<uint32_t>(),
                                                    sys->row_ptr.as<uint32_t>(), (int64_t)M);
      MCS_LAUNCHED();
      if (weights) {
        MCS_TRY(sys->csr_wq.alloc(nu * sizeof(uint64_t), s));
        count_launch();
        gather_entries_kernel<<<grid_for(nu), 256, 0, s>>>(tc, nu, went.as<WEntry>(), sys->csr_cnt.as<uint32_t>(),
                                                           sys->csr_wq.as<uint64_t>());
        MCS_LAUNCHED();
      } else {
        MCS_CUDA(cudaMemcpyAsync(sys->csr_cnt.p, tc, nu * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
      }
    } else {
      MCS_CUDA(cudaMemsetAsync(sys->row_ptr.p, 0, (M + 1) * sizeof(uint32_t), s));
      if (weights) MCS_TRY(sys->csr_wq.alloc(sizeof(uint64_t), s));
    }
  }
  tkeys.release();
  went.release();

  return MC_OK;
}

int assemble_system(mc_system *sys, DevBuf &keys, int64_t n, cudaStream_t s, const uint64_t *weights) {
  const uint64_t N = (uint64_t)sys->n_cols;
  // n_v and 1/n_v
  MCS_TRY(sys->n_v.alloc(N * sizeof(uint32_t), s));
  MCS_TRY(sys->inv_n.alloc(N * sizeof(float), s));
  count_launch(); histories_per_voxel_kernel<<<grid_for((int64_t)N), 256, 0, s>>>(sys->first, sys->count, N, sys->n_v.as<uint32_t>(),
                                                                   sys->inv_n.as<float>());
  MCS_LAUNCHED();
  sys->weighted = weights != nullptr;

  // 1-4. the CSC and CSR: by buckets where columns and rows are short, else
  // by a radix sort
  bool bucketed = false;
  if (!weights && n > 0 && n < ((int64_t)1 << 31)) MCS_TRY(assemble_buckets(sys, keys.as<uint64_t>(), n, s, &bucketed));
  if (bucketed) keys.release();
  else MCS_TRY(assemble_radix(sys, keys, n, s, weights));

  // 5. column sums S_v and the largest count
  {
    MCS_TRY(sys->colsum.alloc(N * sizeof(double), s));
    MCS_TRY(sys->inv_colsum.alloc(N * sizeof(float), s));
    DevBuf mx;
    MCS_TRY(mx.alloc(sizeof(unsigned int), s));
    MCS_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned int), s));
    count_launch(); column_sums_kernel<<<grid_for((int64_t)N), 256, 0, s>>>(sys->col_ptr.as<uint32_t>(), sys->csc_cnt.as<uint32_t>(),
                                                            (int64_t)N, sys->colsum.as<double>(),
                                                            sys->inv_colsum.as<float>(), mx.as<unsigned int>());
    MCS_LAUNCHED();
    if (weights) {
      // S_v from the weights (the kernel above gave the largest event count)
      count_launch();
      column_weight_sums_kernel<<<grid_for((int64_t)N), 256, 0, s>>>(sys->col_ptr.as<uint32_t>(),
                                                                     sys->csc_wq.as<uint64_t>(), (int64_t)N,
                                                                     sys->colsum.as<double>(),
                                                                     sys->inv_colsum.as<float>());
      MCS_LAUNCHED();
    }
    unsigned int mxh = 0;
    MCS_CUDA(cudaMemcpyAsync(&mxh, mx.p, sizeof(mxh), cudaMemcpyDeviceToHost, s));
    MCS_CUDA(cudaStreamSynchronize(s));
    sys->max_count = mxh;
  }
  return MC_OK;
}

// ---------------------------------------------------------------------------
// projector values: the counts in the storage type of sys->value_type
// ---------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V from_count(uint32_t c);
template <> __device__ __forceinline__ float from_count<float>(uint32_t c) { return (float)c; }
template <> __device__ __forceinline__ __half from_count<__half>(uint32_t c) { return __uint2half_rn(c); }
template <> __device__ __forceinline__ __nv_bfloat16 from_count<__nv_bfloat16>(uint32_t c) {
  return __uint2bfloat16_rn(c);
}

template <typename V> __global__ void convert_counts_kernel(const uint32_t *cnt, int64_t n, V *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = from_count<V>(cnt[i]);
}

// weighted systems: the fixed-point weight sums as float, rounded once from
// the integer and scaled by 2^-48 exactly (the same value as a conversion
// through double for sums below 2^53, without the slow FP64 unit)
__global__ void convert_weights_kernel(const uint64_t *wq, int64_t n, float *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __ull2float_rn(wq[i]) * (float)(1.0 / kFdScale);
}

// rounded-A values: val = round(C_jv / n_v) per entry of the CSR (column
// index per entry) ...
template <typename V> __device__ __forceinline__ V from_double(double a);
template <> __device__ __forceinline__ __half from_double<__half>(double a) { return __double2half(a); }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double a) {
  return __double2bfloat16(a);
}
template <typename V>
__global__ void a_values_csr_kernel(const uint32_t *cnt, const uint32_t *col, const uint32_t *n_v, int64_t n, V *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = from_double<V>((double)cnt[i] / (double)n_v[col[i]]);
}
// ... and per column of the CSC, with the column sums of the stored values
// (the rounded matrix's sensitivity s~_v, summed in double in row order)
template <typename V>
__global__ void a_values_csc_kernel(const uint32_t *col_ptr, const uint32_t *cnt, const uint32_t *n_v, int64_t n_cols,
                                    V *out, float *ones, double *sens, float *inv_sens) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_cols; v += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    const double nv = (double)n_v[v];
    for (uint32_t k = col_ptr[v]; k < col_ptr[v + 1]; ++k) {
      const V a = from_double<V>((double)cnt[k] / nv);
      out[k] = a;
      acc += (double)(float)a;
    }
    ones[v] = 1.0f;
    sens[v] = acc;
    inv_sens[v] = acc > 0.0 ? (float)(1.0 / acc) : 0.0f;
  }
}

// counts rounded to V: the column sums of the stored (rounded) counts
template <typename V>
__global__ void rounded_count_sums_kernel(const uint32_t *col_ptr, const uint32_t *cnt, int64_t n_cols, double *sums,
                                          float *inv_sums) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_cols; v += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (uint32_t k = col_ptr[v]; k < col_ptr[v + 1]; ++k) acc += (double)(float)from_count<V>(cnt[k]);
    sums[v] = acc;
    inv_sums[v] = acc > 0.0 ? (float)(1.0 / acc) : 0.0f;
  }
}

template <typename V> static int make_rounded_sums(mc_system *sys, cudaStream_t s) {
  const int64_t N = sys->n_cols;
  const size_t nb = (size_t)(N > 0 ? N : 1);
  MCS_TRY(sys->a_sens.alloc(nb * sizeof(double), s));
  MCS_TRY(sys->a_inv_sens.alloc(nb * sizeof(float), s));
  if (N > 0) {
    count_launch();
    rounded_count_sums_kernel<V><<<grid_for(N), 256, 0, s>>>(sys->col_ptr.as<uint32_t>(), sys->csc_cnt.as<uint32_t>(),
                                                             N, sys->a_sens.as<double>(), sys->a_inv_sens.as<float>());
  }
  MCS_LAUNCHED();
  return MC_OK;
}

template <typename V> static int make_a_values(mc_system *sys, cudaStream_t s) {
  const int64_t nnz = sys->nnz, N = sys->n_cols;
  const size_t nb = (size_t)(N > 0 ? N : 1);
  MCS_TRY(sys->a_ones.alloc(nb * sizeof(float), s));
  MCS_TRY(sys->a_sens.alloc(nb * sizeof(double), s));
  MCS_TRY(sys->a_inv_sens.alloc(nb * sizeof(float), s));
  if (nnz > 0) {
    count_launch();
    a_values_csr_kernel<V><<<grid_for(nnz), 256, 0, s>>>(sys->csr_cnt.as<uint32_t>(), sys->col_idx.as<uint32_t>(),
                                                         sys->n_v.as<uint32_t>(), nnz, sys->csr_val.as<V>());
  }
  if (N > 0) {
    count_launch();
    a_values_csc_kernel<V><<<grid_for(N), 256, 0, s>>>(sys->col_ptr.as<uint32_t>(), sys->csc_cnt.as<uint32_t>(),
                                                       sys->n_v.as<uint32_t>(), N, sys->csc_val.as<V>(),
                                                       sys->a_ones.as<float>(), sys->a_sens.as<double>(),
                                                       sys->a_inv_sens.as<float>());
  }
  MCS_LAUNCHED();
  return MC_OK;
}

int make_values(mc_system *sys, cudaStream_t s) {
  const int64_t nnz = sys->nnz;
  const size_t es = value_storage(sys->value_type) == 0 ? 4 : 2;
  const size_t bytes = (size_t)(nnz > 0 ? nnz : 1) * es;
  MCS_TRY(sys->csr_val.alloc(bytes, s));
  MCS_TRY(sys->csc_val.alloc(bytes, s));
  if (sys->weighted && sys->value_type != MC_VAL_F32) { set_error("weighted systems keep float values"); return MC_EINVAL; }
  if (sys->value_type == MC_VAL_F16_A) return make_a_values<__half>(sys, s);
  if (sys->value_type == MC_VAL_BF16_A) return make_a_values<__nv_bfloat16>(sys, s);
  // counts beyond the type's exact range are rounded: normalise with the
  // rounded counts' column sums
  sys->rounded_counts = (sys->value_type == MC_VAL_F16 && sys->max_count > 2048u) ||
                        (sys->value_type == MC_VAL_BF16 && sys->max_count > 256u);
  if (sys->rounded_counts) {
    if (sys->value_type == MC_VAL_F16) MCS_TRY(make_rounded_sums<__half>(sys, s));
    else MCS_TRY(make_rounded_sums<__nv_bfloat16>(sys, s));
  }
  if (nnz == 0) return MC_OK;
  const int g = grid_for(nnz);
  if (sys->weighted) {
    count_launch(); convert_weights_kernel<<<g, 256, 0, s>>>(sys->csr_wq.as<uint64_t>(), nnz, sys->csr_val.as<float>());
    count_launch(); convert_weights_kernel<<<g, 256, 0, s>>>(sys->csc_wq.as<uint64_t>(), nnz, sys->csc_val.as<float>());
  } else if (sys->value_type == MC_VAL_F32) {
    count_launch(); convert_counts_kernel<float><<<g, 256, 0, s>>>(sys->csr_cnt.as<uint32_t>(), nnz, sys->csr_val.as<float>());
    count_launch(); convert_counts_kernel<float><<<g, 256, 0, s>>>(sys->csc_cnt.as<uint32_t>(), nnz, sys->csc_val.as<float>());
  } else if (sys->value_type == MC_VAL_F16) {
    count_launch(); convert_counts_kernel<__half><<<g, 256, 0, s>>>(sys->csr_cnt.as<uint32_t>(), nnz, sys->csr_val.as<__half>());
    count_launch(); convert_counts_kernel<__half><<<g, 256, 0, s>>>(sys->csc_cnt.as<uint32_t>(), nnz, sys->csc_val.as<__half>());
  } else {
    count_launch(); convert_counts_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(sys->csr_cnt.as<uint32_t>(), nnz,
                                                           sys->csr_val.as<__nv_bfloat16>());
    count_launch(); convert_counts_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(sys->csc_cnt.as<uint32_t>(), nnz,
                                                           sys->csc_val.as<__nv_bfloat16>());
  }
  MCS_LAUNCHED();
  return MC_OK;
}

}  // namespace mcs

// ---------------------------------------------------------------------------
// subset systems (ordered subsets of views, Sec. 5.3)
// ---------------------------------------------------------------------------
namespace mcs {

// row i of the subset = row map[i] of the parent: view subset + (i / rpv) * n_sub
__global__ void subset_rows_kernel(int64_t m_s, int64_t rpv, int n_sub, int subset, const uint32_t *parent_ptr,
                                   uint32_t *map, uint32_t *len) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_s; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t view = subset + (i / rpv) * n_sub;
    const uint32_t r = (uint32_t)(view * rpv + i % rpv);
    map[i] = r;
    len[i] = parent_ptr[r + 1] - parent_ptr[r];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) len[m_s] = 0u;
}

// copy the parent's entries of each subset row; emit (col * m_s + i, count)
__global__ void subset_copy_kernel(int64_t m_s, const uint32_t *map, const uint32_t *parent_ptr,
                                   const uint32_t *parent_col, const uint32_t *parent_cnt, const uint32_t *ptr,
                                   uint32_t *col, uint32_t *cnt, uint64_t *tkeys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_s; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t src = parent_ptr[map[i]], dst = ptr[i], n = ptr[i + 1] - ptr[i];
    for (uint32_t k = 0; k < n; ++k) {
      const uint32_t c = parent_col[src + k];
      col[dst + k] = c;
      cnt[dst + k] = parent_cnt[src + k];
      tkeys[dst + k] = (uint64_t)c * (uint64_t)m_s + (uint64_t)i;
    }
  }
}

__global__ void sum_counts_kernel(const uint32_t *cnt, int64_t n, unsigned long long *out) {
  unsigned long long acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += cnt[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

int subset_system(const mc_system *parent, int64_t rpv, int n_sub, int subset, mc_system *sys, cudaStream_t s) {
  const int64_t V = parent->n_rows / rpv;
  const int64_t nv_s = (V - subset + n_sub - 1) / n_sub;
  const int64_t m_s = nv_s * rpv, N = parent->n_cols;
  sys->n_rows = m_s;
  sys->n_cols = N;
  sys->first = parent->first;
  sys->count = parent->count;
  sys->parent_rows = parent->n_rows;
  sys->n_subsets = n_sub;
  sys->subset = subset;
  MCS_TRY(sys->row_map.alloc((size_t)m_s * sizeof(uint32_t), s));
  DevBuf len;
  MCS_TRY(len.alloc((size_t)(m_s + 1) * sizeof(uint32_t), s));
  MCS_TRY(sys->row_ptr.alloc((size_t)(m_s + 1) * sizeof(uint32_t), s));
  count_launch();
  subset_rows_kernel<<<grid_for(m_s), 256, 0, s>>>(m_s, rpv, n_sub, subset, parent->row_ptr.as<uint32_t>(),
                                                  sys->row_map.as<uint32_t>(), len.as<uint32_t>());
  MCS_LAUNCHED();
  MCS_TRY(exclusive_scan_u32(len.as<uint32_t>(), sys->row_ptr.as<uint32_t>(), m_s + 1, s));
  uint32_t nnz = 0;
  MCS_CUDA(cudaMemcpyAsync(&nnz, sys->row_ptr.as<uint32_t>() + m_s, 4, cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  sys->nnz = nnz;
  const size_t nb = (size_t)(nnz > 0 ? nnz : 1);
  DevBuf tkeys, tkeys_alt, tcnt, tcnt_alt;
  MCS_TRY(sys->col_idx.alloc(nb * 4, s));
  MCS_TRY(sys->csr_cnt.alloc(nb * 4, s));
  MCS_TRY(tkeys.alloc(nb * 8, s));
  MCS_TRY(tkeys_alt.alloc(nb * 8, s));
  MCS_TRY(tcnt.alloc(nb * 4, s));
  MCS_TRY(tcnt_alt.alloc(nb * 4, s));
  count_launch();
  subset_copy_kernel<<<grid_for(m_s), 256, 0, s>>>(m_s, sys->row_map.as<uint32_t>(), parent->row_ptr.as<uint32_t>(),
                                                  parent->col_idx.as<uint32_t>(), parent->csr_cnt.as<uint32_t>(),
                                                  sys->row_ptr.as<uint32_t>(), sys->col_idx.as<uint32_t>(),
                                                  sys->csr_cnt.as<uint32_t>(), tkeys.as<uint64_t>());
  MCS_LAUNCHED();
  // CSC of the subset: sort (col * m_s + row, count)
  MCS_CUDA(cudaMemcpyAsync(tcnt.p, sys->csr_cnt.p, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
  bool alt = false;
  MCS_TRY(radix_sort_u64(tkeys.as<uint64_t>(), tkeys_alt.as<uint64_t>(), tcnt.as<uint32_t>(), tcnt_alt.as<uint32_t>(),
                         nnz, bits_for((uint64_t)m_s * (uint64_t)N - 1), &alt, s));
  const uint64_t *tk = alt ? tkeys_alt.as<uint64_t>() : tkeys.as<uint64_t>();
  const uint32_t *tc = alt ? tcnt_alt.as<uint32_t>() : tcnt.as<uint32_t>();
  DevBuf hist;
  MCS_TRY(hist.alloc((size_t)(N + 1) * 4, s));
  MCS_CUDA(cudaMemsetAsync(hist.p, 0, (size_t)(N + 1) * 4, s));
  MCS_TRY(sys->col_ptr.alloc((size_t)(N + 1) * 4, s));
  MCS_TRY(sys->row_idx.alloc(nb * 4, s));
  MCS_TRY(sys->csc_cnt.alloc(nb * 4, s));
  if (nnz > 0) {
    count_launch();
    split_keys_kernel<<<grid_for(nnz), 256, 0, s>>>(tk, nnz, (uint64_t)m_s, nullptr, sys->row_idx.as<uint32_t>(),
                                                    hist.as<uint32_t>());
    MCS_LAUNCHED();
    MCS_CUDA(cudaMemcpyAsync(sys->csc_cnt.p, tc, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
  }
  MCS_TRY(exclusive_scan_u32(hist.as<uint32_t>(), sys->col_ptr.as<uint32_t>(), N + 1, s));
  // histories per voxel are the parent's; column sums and largest count
  MCS_TRY(sys->n_v.alloc((size_t)N * 4, s));
  MCS_TRY(sys->inv_n.alloc((size_t)N * 4, s));
  MCS_CUDA(cudaMemcpyAsync(sys->n_v.p, parent->n_v.p, (size_t)N * 4, cudaMemcpyDeviceToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(sys->inv_n.p, parent->inv_n.p, (size_t)N * 4, cudaMemcpyDeviceToDevice, s));
  MCS_TRY(sys->colsum.alloc((size_t)N * sizeof(double), s));
  MCS_TRY(sys->inv_colsum.alloc((size_t)N * sizeof(float), s));
  DevBuf mx;
  MCS_TRY(mx.alloc(2 * sizeof(unsigned long long), s));
  MCS_CUDA(cudaMemsetAsync(mx.p, 0, 2 * sizeof(unsigned long long), s));
  count_launch();
  column_sums_kernel<<<grid_for(N), 256, 0, s>>>(sys->col_ptr.as<uint32_t>(), sys->csc_cnt.as<uint32_t>(), N,
                                                 sys->colsum.as<double>(), sys->inv_colsum.as<float>(),
                                                 mx.as<unsigned int>());
  count_launch();
  sum_counts_kernel<<<grid_for(nnz > 0 ? nnz : 1), 256, 0, s>>>(sys->csr_cnt.as<uint32_t>(), nnz,
                                                                mx.as<unsigned long long>() + 1);
  MCS_LAUNCHED();
  unsigned long long h[2] = {0, 0};
  MCS_CUDA(cudaMemcpyAsync(h, mx.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  sys->max_count = (uint32_t)(h[0] & 0xFFFFFFFFull);
  sys->n_events = (int64_t)h[1];
  for (int f = 0; f < 4; ++f) sys->fates[f] = parent->fates[f];
  return MC_OK;
}

}  // namespace mcs
