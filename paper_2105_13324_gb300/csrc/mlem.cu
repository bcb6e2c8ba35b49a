// mlem.cu -- projectors and the ML-EM update (paper Sec. 5.1, Eq. (IMC) and
// Eq. (MLEM)).
//
// The system is stored as integer counts C_jv with A = C diag(1/n_v), n_v
// the histories started in voxel v.  With xs_v = x_v / n_v:
//   forward      q_j = sum_v C_jv xs_v                      (CSR gather)
//   ratio        r_j = y_j / q_j, 0 where q_j = 0
//   back + EM    x_v <- x_v * (sum_j C_jv r_j) / S_v,  S_v = sum_j C_jv
// (the 1/n_v of the back-projection and of the sensitivity s_v = S_v / n_v
// cancel in the update).  Both halves are gathers over the explicitly stored
// CSR and CSC, so no floating-point atomics are used and the result is the
// same from run to run.  Each row (column) is reduced by a group of G lanes,
// G a power of two matched to the mean row (column) length.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

namespace mcs {

constexpr int kSpmvThreads = 256;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

__global__ void prescale_kernel(const float *x, const float *inv_n, float *xs, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xs[i] = x[i] * inv_n[i];
}

// Sum of a double over the block (fixed order); valid in thread 0.
__device__ __forceinline__ double block_sum_double(double v, double *s_tmp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_tmp[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
  __syncthreads();
  return t;
}

// Partial sum, for lane `sub` of a group of G lanes, of val[k] * vec[idx[k]]
// over k in [b, e).  The matrix streams are read with 16-byte vector loads
// (4 entries per lane per step) between a scalar head that reaches a
// multiple of 4 and a scalar tail, and with the streaming cache hint so that
// they do not evict the gathered vector from L2.
__device__ __forceinline__ void load4(const float *p, float v[4]) {
  const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const __half *p, float v[4]) {
  const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
  const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load4(const __nv_bfloat16 *p, float v[4]) {
  const uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&t.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename V, int G>
__device__ __forceinline__ float segment_dot(uint32_t b, uint32_t e, const uint32_t *__restrict__ idx,
                                             const V *__restrict__ val, const float *__restrict__ vec, int sub) {
  float acc = 0.0f;
  uint32_t a = (b + 3u) & ~3u;
  if (a > e) a = e;
  for (uint32_t k = b + sub; k < a; k += G) acc = fmaf(to_f(__ldcs(val + k)), __ldg(vec + __ldcs(idx + k)), acc);
  const uint32_t t = a + ((e - a) & ~3u);
  uint32_t k = a + 4u * sub;
  // two 4-entry vectors per lane per step: both loads issue before the gathers
  for (; k + 4u * G < t; k += 8u * G) {
    const uint4 i4 = __ldcs(reinterpret_cast<const uint4 *>(idx + k));
    const uint4 j4 = __ldcs(reinterpret_cast<const uint4 *>(idx + k + 4u * G));
    float v[4], w[4];
    load4(val + k, v);
    load4(val + k + 4u * G, w);
    acc = fmaf(v[0], __ldg(vec + i4.x), acc);
    acc = fmaf(v[1], __ldg(vec + i4.y), acc);
    acc = fmaf(v[2], __ldg(vec + i4.z), acc);
    acc = fmaf(v[3], __ldg(vec + i4.w), acc);
    acc = fmaf(w[0], __ldg(vec + j4.x), acc);
    acc = fmaf(w[1], __ldg(vec + j4.y), acc);
    acc = fmaf(w[2], __ldg(vec + j4.z), acc);
    acc = fmaf(w[3], __ldg(vec + j4.w), acc);
  }
  for (; k < t; k += 4u * G) {
    const uint4 i4 = __ldcs(reinterpret_cast<const uint4 *>(idx + k));
    float v[4];
    load4(val + k, v);
    acc = fmaf(v[0], __ldg(vec + i4.x), acc);
    acc = fmaf(v[1], __ldg(vec + i4.y), acc);
    acc = fmaf(v[2], __ldg(vec + i4.z), acc);
    acc = fmaf(v[3], __ldg(vec + i4.w), acc);
  }
  for (uint32_t k = t + sub; k < e; k += G) acc = fmaf(to_f(__ldcs(val + k)), __ldg(vec + __ldcs(idx + k)), acc);
  return acc;
}

// MODE 0: out = q.  MODE 1: out = r = y / q (0 where q = 0), and with LL the
// block's share of sum_j (y_j ln q_j - q_j) in partials[blockIdx.x].
// MODE 2: r_i = y_o / (q_i + add_o), o = rmap[i] (i without a map), 0 where
// the denominator is not positive (Eq. (Sohlberg OSEM) of Sec. 5.4).
template <int MODE>
__device__ __forceinline__ float ratio_out(float acc, int64_t i, const float *y, const uint32_t *rmap, const float *add) {
  if (MODE == 1) {
    const float yj = y[i];
    return acc > 0.0f ? yj / acc : 0.0f;
  }
  const int64_t o = rmap ? (int64_t)rmap[i] : i;
  const float den = acc + (add ? add[o] : 0.0f);
  return den > 0.0f ? y[o] / den : 0.0f;
}

template <typename V, int G, int MODE, bool LL>
__global__ void __launch_bounds__(kSpmvThreads) csr_forward_kernel(const uint32_t *__restrict__ row_ptr,
                                                                   const uint32_t *__restrict__ col,
                                                                   const V *__restrict__ val,
                                                                   const float *__restrict__ xs, int64_t m,
                                                                   const float *__restrict__ y,
                                                                   float *__restrict__ out, double *partials,
                                                                   const uint32_t *__restrict__ rmap,
                                                                   const float *__restrict__ add) {
  __shared__ double s_tmp[kSpmvThreads / 32];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t gid = ((int64_t)blockIdx.x * kSpmvThreads + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  double ll = 0.0;
  // every lane takes part in the shuffles; lanes past the last row see an
  // empty range
  uint32_t b = 0, e = 0;
  float yv = 0.0f;  // the ratio's y, issued ahead of the gathers
  if (gid < m) {
    b = row_ptr[gid];
    e = row_ptr[gid + 1];
    if (MODE == 1 && sub == 0) yv = y[gid];
  }
  float acc = segment_dot<V, G>(b, e, col, val, xs, sub);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
  if (gid < m && sub == 0) {
    if (MODE == 0) {
      out[gid] = acc;
    } else {
      out[gid] = MODE == 1 ? (acc > 0.0f ? yv / acc : 0.0f) : ratio_out<MODE>(acc, gid, y, rmap, add);
      if (LL) {
        // a bin with an empty row is left out of the y ln q sum (q = 0 for
        // every image: the term carries no information about x)
        const float yj = MODE == 1 ? yv : y[gid];
        ll = (yj > 0.0f && e > b ? (double)yj * log((double)acc) : 0.0) - (double)acc;
      }
    }
  }
  if (LL) {
    const double t = block_sum_double(ll, s_tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// MODE 0: out_v = (1/n_v) sum_j C_jv r_j (back-projection A^T r).
// MODE 1: x_v <- x_v t_v / S_v (0 where S_v = 0), xs_v = x_v / n_v.
// MODE 3: as MODE 1 but x_v is kept where S_v = 0 (a voxel outside an
// ordered subset's view is not updated by that subset).
template <typename V, int G, int MODE>
__global__ void __launch_bounds__(kSpmvThreads) csc_back_kernel(const uint32_t *__restrict__ col_ptr,
                                                                const uint32_t *__restrict__ row,
                                                                const V *__restrict__ val,
                                                                const float *__restrict__ r, int64_t n,
                                                                const float *__restrict__ inv_n,
                                                                const float *__restrict__ inv_colsum,
                                                                float *__restrict__ x, float *__restrict__ xs) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t gid = ((int64_t)blockIdx.x * kSpmvThreads + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  uint32_t b = 0, e = 0;
  // the epilogue's loads are issued with the pointers, ahead of the gathers
  float is = 0.0f, xv = 0.0f, in = 0.0f;
  if (gid < n) {
    b = col_ptr[gid];
    e = col_ptr[gid + 1];
    if (sub == 0) {
      in = inv_n[gid];
      if (MODE != 0) {
        is = inv_colsum[gid];
        xv = x[gid];
      }
    }
  }
  float acc = segment_dot<V, G>(b, e, row, val, r, sub);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
  if (gid < n && sub == 0) {
    if (MODE == 0) {
      x[gid] = acc * in;
    } else {
      const float xn = is > 0.0f ? xv * acc * is : (MODE == 3 ? xv : 0.0f);
      x[gid] = xn;
      xs[gid] = xn * in;
    }
  }
}

__global__ void sum_partials_kernel(const double *partials, int64_t n, double *out) {
  __shared__ double s_tmp[32];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  const double t = block_sum_double(acc, s_tmp);
  if (threadIdx.x == 0) *out = t;
}

// partials[b] = block b's sum of y (double) and of s_v = S_v / n_v (n_v
// NULL: colsum holds s_v itself)
__global__ void init_sums_kernel(const float *y, int64_t m, const double *colsum, const uint32_t *n_v, int64_t n,
                                 double *py, double *ps) {
  __shared__ double s_tmp[32];
  double ay = 0.0, as = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    ay += (double)y[i];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (!n_v) as += colsum[v];
    else if (n_v[v]) as += colsum[v] / (double)n_v[v];
  }
  const double ty = block_sum_double(ay, s_tmp);
  const double ts = block_sum_double(as, s_tmp);
  if (threadIdx.x == 0) { py[blockIdx.x] = ty; ps[blockIdx.x] = ts; }
}

// x0 = sum(y) / sum(s) from the block partials (one block, fixed order)
__global__ void init_total_kernel(const double *py, const double *ps, int nb, double *x0) {
  __shared__ double s_tmp[32];
  double ay = 0.0, as = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) { ay += py[b]; as += ps[b]; }
  const double sy = block_sum_double(ay, s_tmp);
  const double ss = block_sum_double(as, s_tmp);
  if (threadIdx.x == 0) *x0 = ss > 0.0 ? sy / ss : 0.0;
}

__global__ void init_fill_kernel(const double *x0p, const double *colsum, const float *inv_n, int64_t n, float *x,
                                 float *xs) {
  const float x0 = (float)*x0p;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float xv = colsum[v] > 0.0 ? x0 : 0.0f;
    x[v] = xv;
    xs[v] = xv * inv_n[v];
  }
}

__global__ void sensitivity_kernel(const double *colsum, const uint32_t *n_v, int64_t n, double *s) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    s[v] = !n_v ? colsum[v] : n_v[v] ? colsum[v] / (double)n_v[v] : 0.0;
}

// ---------------------------------------------------------------------------
// streaming SpMV: one block per tile of at most kStreamTile non-zeros
// ---------------------------------------------------------------------------
// A tile is a run of whole rows (columns) whose entries are contiguous in the
// CSR (CSC) arrays.  The block first reads the tile's entries and gathers the
// vector with independent, coalesced loads (many requests in flight), keeps
// the products in shared memory, and then reduces each row from shared
// memory: one warp per row (segments of 16 or more entries on average), or
// one thread per row (the batch kernels).  Single systems with shorter
// segments use the warp chunks below instead.  Every row is summed in a fixed
// order, so results are reproducible.
constexpr int kStreamTile = 4096;
constexpr int kStreamThreads = 256;

// Products of the tile's entries [p0, p0 + cnt) into s_prod.  The index
// and value streams are read as aligned quads (16-byte index loads, two
// quads per thread in flight); the partial quads at the two ends of the
// tile take scalar loads.
template <typename V>
__device__ __forceinline__ void stream_products(uint32_t p0, uint32_t cnt, const uint32_t *__restrict__ idx,
                                                const V *__restrict__ val, const float *__restrict__ vec,
                                                float *s_prod) {
  const uint32_t h = p0 & 3u;                  // entries of the first quad before p0
  const uint32_t nq = (h + cnt + 3u) >> 2;      // quads covering [p0 - h, p0 + cnt)
  const uint32_t base = p0 - h;
#pragma unroll 2
  for (uint32_t q = threadIdx.x; q < nq; q += kStreamThreads) {
    const int32_t i0 = (int32_t)(4u * q) - (int32_t)h;  // tile offset of the quad's first entry
    if (i0 >= 0 && i0 + 4 <= (int32_t)cnt) {
      const uint4 c = __ldcs(reinterpret_cast<const uint4 *>(idx + base) + q);
      float v[4];
      load4(val + base + 4u * q, v);
      s_prod[i0] = v[0] * __ldg(vec + c.x);
      s_prod[i0 + 1] = v[1] * __ldg(vec + c.y);
      s_prod[i0 + 2] = v[2] * __ldg(vec + c.z);
      s_prod[i0 + 3] = v[3] * __ldg(vec + c.w);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t i = i0 + u;
        if (i >= 0 && i < (int32_t)cnt) s_prod[i] = to_f(__ldcs(val + p0 + i)) * __ldg(vec + __ldcs(idx + p0 + i));
      }
    }
  }
}

// Sum of the products of segment [b, e) of the tile: one thread, or the 32
// lanes of a warp (result in every lane).
template <bool WARP>
__device__ __forceinline__ float stream_segment(const float *s_prod, uint32_t b, uint32_t e) {
  float acc = 0.0f;
  if (WARP) {
    for (uint32_t k = b + (threadIdx.x & 31); k < e; k += 32) acc += s_prod[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  } else {
    for (uint32_t k = b; k < e; ++k) acc += s_prod[k];
  }
  return acc;
}

// Reduces every segment j in [j0, j1) of the tile from shared memory and
// hands its sum to out.store(j, acc, out.load(j), segment j non-empty).  Warp
// mode: one warp per
// segment.  Thread mode: each thread takes kSegBatch segments kStreamThreads
// apart and issues their pointer loads and out.load() before any reduction,
// so that short segments do not leave one load in flight per thread.
constexpr int kSegBatch = 4;
template <typename Out>
__device__ __forceinline__ void stream_segments_thread(const uint32_t *__restrict__ ptr, uint32_t j0, uint32_t j1,
                                                       uint32_t p0, const float *s_prod, Out &out) {
  for (uint32_t base = j0 + threadIdx.x; base < j1; base += kSegBatch * kStreamThreads) {
    uint32_t b[kSegBatch], e[kSegBatch];
    typename Out::Pre pre[kSegBatch] = {};
#pragma unroll
    for (int u = 0; u < kSegBatch; ++u) {
      const uint32_t j = base + u * kStreamThreads;
      b[u] = e[u] = p0;
      if (j < j1) {
        b[u] = ptr[j];
        e[u] = ptr[j + 1];
        pre[u] = out.load(j);
      }
    }
#pragma unroll
    for (int u = 0; u < kSegBatch; ++u) {
      const uint32_t j = base + u * kStreamThreads;
      if (j < j1) out.store(j, stream_segment<false>(s_prod, b[u] - p0, e[u] - p0), pre[u], e[u] > b[u]);
    }
  }
}

template <bool WARP, typename Out>
__device__ __forceinline__ void stream_segments(const uint32_t *__restrict__ ptr, uint32_t j0, uint32_t j1,
                                                uint32_t p0, const float *s_prod, Out &out) {
  if (WARP) {
    for (uint32_t j = j0 + (threadIdx.x >> 5); j < j1; j += kStreamThreads / 32) {
      const uint32_t b = ptr[j], e = ptr[j + 1];
      const float acc = stream_segment<true>(s_prod, b - p0, e - p0);
      if ((threadIdx.x & 31) == 0) out.store(j, acc, out.load(j), e > b);
    }
  } else {
    stream_segments_thread(ptr, j0, j1, p0, s_prod, out);
  }
}

// Forward epilogue: MODE 0 q, MODE 1 ratio (+ log-likelihood share),
// MODE 2 ratio with row map and additive term (see ratio_out).
template <int MODE, bool LL>
struct FwdOut {
  using Pre = float;
  const float *__restrict__ y;
  float *__restrict__ out;
  const uint32_t *__restrict__ rmap;
  const float *__restrict__ add;
  double ll;
  __device__ __forceinline__ float load(uint32_t r) const { return (MODE == 1) ? y[r] : 0.0f; }
  // `reached`: the row holds an entry (a bin with an empty row is left out
  // of the y ln q sum)
  __device__ __forceinline__ void store(uint32_t r, float acc, float yv, bool reached) {
    if (MODE == 0) {
      out[r] = acc;
    } else if (MODE == 1) {
      out[r] = acc > 0.0f ? yv / acc : 0.0f;
      if (LL) ll += (yv > 0.0f && reached ? (double)yv * log((double)acc) : 0.0) - (double)acc;
    } else {
      out[r] = ratio_out<MODE>(acc, r, y, rmap, add);
    }
  }
};

// Back-projection epilogue: MODE 0 A^T r, MODE 1 EM update (0 where S = 0),
// MODE 3 EM update keeping x where S = 0.
struct BackPre { float is, x, inv_n; };
template <int MODE>
struct BackOut {
  using Pre = BackPre;
  const float *__restrict__ inv_n;
  const float *__restrict__ inv_colsum;
  float *__restrict__ x;
  float *__restrict__ xs;
  __device__ __forceinline__ BackPre load(uint32_t v) const {
    BackPre p;
    p.inv_n = inv_n[v];
    p.is = MODE == 0 ? 0.0f : inv_colsum[v];
    p.x = MODE == 0 ? 0.0f : x[v];
    return p;
  }
  __device__ __forceinline__ void store(uint32_t v, float acc, const BackPre &p, bool) const {
    if (MODE == 0) {
      x[v] = acc * p.inv_n;
    } else {
      const float xn = p.is > 0.0f ? p.x * acc * p.is : (MODE == 3 ? p.x : 0.0f);
      x[v] = xn;
      xs[v] = xn * p.inv_n;
    }
  }
};

template <typename V, bool WARP, int MODE, bool LL>
__global__ void __launch_bounds__(kStreamThreads) stream_forward_kernel(const uint32_t *__restrict__ row_ptr,
                                                                     const uint32_t *__restrict__ tiles,
                                                                     const uint32_t *__restrict__ col,
                                                                     const V *__restrict__ val,
                                                                     const float *__restrict__ xs,
                                                                     const float *__restrict__ y,
                                                                     float *__restrict__ out, double *partials,
                                                                     const uint32_t *__restrict__ rmap,
                                                                     const float *__restrict__ add) {
  __shared__ float s_prod[kStreamTile];
  __shared__ double s_tmp[kStreamThreads / 32];
  const uint32_t r0 = tiles[blockIdx.x], r1 = tiles[blockIdx.x + 1];
  const uint32_t p0 = row_ptr[r0];
  stream_products<V>(p0, row_ptr[r1] - p0, col, val, xs, s_prod);
  __syncthreads();
  FwdOut<MODE, LL> o{y, out, rmap, add, 0.0};
  stream_segments<WARP>(row_ptr, r0, r1, p0, s_prod, o);
  if (LL) {
    const double t = block_sum_double(o.ll, s_tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

template <typename V, bool WARP, int MODE>
__global__ void __launch_bounds__(kStreamThreads) stream_back_kernel(const uint32_t *__restrict__ col_ptr,
                                                                  const uint32_t *__restrict__ tiles,
                                                                  const uint32_t *__restrict__ row,
                                                                  const V *__restrict__ val,
                                                                  const float *__restrict__ r,
                                                                  const float *__restrict__ inv_n,
                                                                  const float *__restrict__ inv_colsum,
                                                                  float *__restrict__ x, float *__restrict__ xs) {
  __shared__ float s_prod[kStreamTile];
  const uint32_t c0 = tiles[blockIdx.x], c1 = tiles[blockIdx.x + 1];
  const uint32_t p0 = col_ptr[c0];
  stream_products<V>(p0, col_ptr[c1] - p0, row, val, r, s_prod);
  __syncthreads();
  BackOut<MODE> o{inv_n, inv_colsum, x, xs};
  stream_segments<WARP>(col_ptr, c0, c1, p0, s_prod, o);
}

// ---------------------------------------------------------------------------
// warp chunks: short segments, one lane per segment, no block barrier
// ---------------------------------------------------------------------------
// A warp takes the 32 R consecutive segments [j0, j0 + 32 R), lane l the
// segments j0 + l + 32 r (r < R), so that pointer loads and result stores
// stay coalesced.  The chunk's entries are contiguous; the warp reads them in
// windows of kChunkWindow (coalesced index and value loads, then one gather
// per entry), keeps the window's products in its own shared-memory row, and
// each lane adds up its segments' parts of the window in entry order.  A
// segment is therefore summed in the same order, from the same products, as
// by a plain loop over its entries, and segments of any length are handled.
// R (1, 2, 4) is chosen so that a chunk holds about 100 entries or more
// (very short segments leave too few gathers in flight per warp otherwise),
// but no larger than keeps 32 warps per SM in the launch (small launches
// need the warps more than the longer chunks).
// Blocks are small so that few warp slots wait for the slowest warp of a
// block.
constexpr int kChunkWindow = 128;
constexpr int kChunkThreads = 128;
static_assert(kStreamTile >= (kStreamThreads / 32) * kChunkWindow, "a tile block's products hold its warps' windows");

// Segments per lane for n segments averaging nnz / n entries, in a launch
// over `launch_segments` segments in all.
inline int chunk_rows_per_lane(int64_t nnz, int64_t n, int64_t launch_segments) {
  int r = (double)nnz >= 3.0 * (double)n ? 1 : (double)nnz >= 1.5 * (double)n ? 2 : 4;
  const int64_t min_warps = (int64_t)device_sm_count() * 32;
  while (r > 1 && launch_segments / (32 * r) < min_warps) r >>= 1;
  return r;
}

// j0: the warp's first segment (a multiple of 32 R); s_w: the warp's
// kChunkWindow floats.
template <int R, typename V, typename Out>
__device__ __forceinline__ void chunk_segments(const uint32_t *__restrict__ ptr, int64_t n_seg,
                                               const uint32_t *__restrict__ idx, const V *__restrict__ val,
                                               const float *__restrict__ vec, float *s_w, Out &out, int64_t j0) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t b[R], e[R];
  typename Out::Pre pre[R];
  float acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t j = j0 + lane + 32 * r;
    const bool mine = j < n_seg;
    b[r] = ptr[mine ? j : n_seg];
    e[r] = ptr[mine ? j + 1 : n_seg];
    pre[r] = typename Out::Pre{};
    if (mine) pre[r] = out.load((uint32_t)j);
    acc[r] = 0.0f;
  }
  // the chunk's entries [p0, p1): lane 0's first to lane 31's last
  const uint32_t p0 = __shfl_sync(0xffffffffu, b[0], 0), p1 = __shfl_sync(0xffffffffu, e[R - 1], 31);
  for (uint32_t w0 = p0; w0 < p1; w0 += kChunkWindow) {
    const uint32_t n = min((uint32_t)kChunkWindow, p1 - w0);
    const uint32_t *ip = idx + w0 + lane;
    const V *vp = val + w0 + lane;
    uint32_t c[kChunkWindow / 32];
    float v[kChunkWindow / 32];
#pragma unroll
    for (int u = 0; u < kChunkWindow / 32; ++u) {
      c[u] = 0u;
      v[u] = 0.0f;
      if (lane + 32u * u < n) {
        c[u] = __ldcs(ip + 32 * u);
        v[u] = to_f(__ldcs(vp + 32 * u));
      }
    }
#pragma unroll
    for (int u = 0; u < kChunkWindow / 32; ++u)
      if (lane + 32u * u < n) s_w[lane + 32 * u] = v[u] * __ldg(vec + c[u]);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t lo = b[r] > w0 ? b[r] : w0, hi = e[r] < w0 + n ? e[r] : w0 + n;
      const uint32_t len = hi > lo ? hi - lo : 0u;
      const float *q = s_w + (len ? lo - w0 : 0u), *qe = q + len;
      float t = acc[r];
      for (; q + 1 < qe; q += 2) { t += q[0]; t += q[1]; }
      if (q < qe) t += q[0];
      acc[r] = t;
    }
    __syncwarp();
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int64_t j = j0 + lane + 32 * r;
    if (j < n_seg) out.store((uint32_t)j, acc[r], pre[r], e[r] > b[r]);
  }
}

// the warp's first segment in the single-system kernels
template <int R> __device__ __forceinline__ int64_t chunk_first() {
  return ((int64_t)blockIdx.x * kChunkThreads + (threadIdx.x & ~31u)) * R;
}

template <int R, typename V, int MODE, bool LL>
__global__ void __launch_bounds__(kChunkThreads) chunk_forward_kernel(const uint32_t *__restrict__ row_ptr, int64_t m,
                                                                   const uint32_t *__restrict__ col,
                                                                   const V *__restrict__ val,
                                                                   const float *__restrict__ xs,
                                                                   const float *__restrict__ y,
                                                                   float *__restrict__ out, double *partials,
                                                                   const uint32_t *__restrict__ rmap,
                                                                   const float *__restrict__ add) {
  __shared__ float s_w[kChunkThreads / 32][kChunkWindow];
  __shared__ double s_tmp[kChunkThreads / 32];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  FwdOut<MODE, LL> o{y, out, rmap, add, 0.0};
  chunk_segments<R, V>(row_ptr, m, col, val, xs, s_w[threadIdx.x >> 5], o, chunk_first<R>());
  if (LL) {
    const double t = block_sum_double(o.ll, s_tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

template <int R, typename V, int MODE>
__global__ void __launch_bounds__(kChunkThreads) chunk_back_kernel(const uint32_t *__restrict__ col_ptr, int64_t n,
                                                                const uint32_t *__restrict__ row,
                                                                const V *__restrict__ val,
                                                                const float *__restrict__ r,
                                                                const float *__restrict__ inv_n,
                                                                const float *__restrict__ inv_colsum,
                                                                float *__restrict__ x, float *__restrict__ xs) {
  __shared__ float s_w[kChunkThreads / 32][kChunkWindow];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  BackOut<MODE> o{inv_n, inv_colsum, x, xs};
  chunk_segments<R, V>(col_ptr, n, row, val, r, s_w[threadIdx.x >> 5], o, chunk_first<R>());
}

// longest segment of a CSR/CSC pointer array
__global__ void max_segment_kernel(const uint32_t *ptr, int64_t n, unsigned int *out) {
  uint32_t mx = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t len = ptr[i + 1] - ptr[i];
    mx = len > mx ? len : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint32_t y2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y2 > mx ? y2 : mx;
  }
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// tiles[b] = first segment i with ptr[i] + i >= b * step (tiles[n_tiles] = n):
// the measure counts entries and segments, so a tile holds at most step +
// longest of the two together.  With step = kStreamTile - longest - 1 every
// tile has fewer than kStreamTile entries and rows, however sparse the
// matrix.
__global__ void tile_bounds_kernel(const uint32_t *ptr, int64_t n, uint32_t step, int64_t n_tiles, uint32_t *tiles) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b <= n_tiles; b += (int64_t)gridDim.x * blockDim.x) {
    if (b == n_tiles) { tiles[b] = (uint32_t)n; continue; }
    const uint64_t target = (uint64_t)b * step;
    int64_t lo = 0, hi = n;  // first i in [0, n] with ptr[i] + i >= target
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((uint64_t)ptr[mid] + (uint64_t)mid >= target) hi = mid; else lo = mid + 1;
    }
    tiles[b] = (uint32_t)lo;
  }
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
// Launch with programmatic stream serialisation: the grid may be scheduled
// while the previous kernel on the stream drains; the projector kernels
// launched this way wait at griddepcontrol.wait, before any memory access,
// until that kernel has completed and its writes are visible, so the order
// of the two is that of a plain launch with the launch latency hidden.
template <typename... P, typename... A>
static void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, args...);
}

static int grid_stride_blocks(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <typename V, int MODE, bool LL>
static void fwd_launch(const mc_system *sys, int g, const float *xs, const float *y, float *out, double *partials,
                       cudaStream_t s, const uint32_t *rmap = nullptr, const float *add = nullptr) {
  const int64_t m = sys->n_rows;
  const int blocks = div_up(m * g, kSpmvThreads);
  const V *val = sys->csr_val.as<V>();
  const uint32_t *rp = sys->row_ptr.as<uint32_t>(), *ci = sys->col_idx.as<uint32_t>();
  switch (g) {
    case 1: count_launch(); launch_pdl(csr_forward_kernel<V, 1, MODE, LL>, blocks, kSpmvThreads, s, rp, ci, val, xs, m, y, out, partials, rmap, add); break;
    case 2: count_launch(); launch_pdl(csr_forward_kernel<V, 2, MODE, LL>, blocks, kSpmvThreads, s, rp, ci, val, xs, m, y, out, partials, rmap, add); break;
    case 4: count_launch(); launch_pdl(csr_forward_kernel<V, 4, MODE, LL>, blocks, kSpmvThreads, s, rp, ci, val, xs, m, y, out, partials, rmap, add); break;
    case 8: count_launch(); launch_pdl(csr_forward_kernel<V, 8, MODE, LL>, blocks, kSpmvThreads, s, rp, ci, val, xs, m, y, out, partials, rmap, add); break;
    case 16: count_launch(); launch_pdl(csr_forward_kernel<V, 16, MODE, LL>, blocks, kSpmvThreads, s, rp, ci, val, xs, m, y, out, partials, rmap, add); break;
    default: count_launch(); launch_pdl(csr_forward_kernel<V, 32, MODE, LL>, blocks, kSpmvThreads, s, rp, ci, val, xs, m, y, out, partials, rmap, add); break;
  }
}

template <typename V, int MODE>
static void back_launch(const mc_system *sys, int g, const float *r, float *x, float *xs, cudaStream_t s) {
  const int64_t n = sys->n_cols;
  const int blocks = div_up(n * g, kSpmvThreads);
  const V *val = sys->csc_val.as<V>();
  const uint32_t *cp = sys->col_ptr.as<uint32_t>(), *ri = sys->row_idx.as<uint32_t>();
  const float *inv_n = proj_scale(sys), *ics = proj_inv_norm(sys);
  switch (g) {
    case 1: count_launch(); launch_pdl(csc_back_kernel<V, 1, MODE>, blocks, kSpmvThreads, s, cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 2: count_launch(); launch_pdl(csc_back_kernel<V, 2, MODE>, blocks, kSpmvThreads, s, cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 4: count_launch(); launch_pdl(csc_back_kernel<V, 4, MODE>, blocks, kSpmvThreads, s, cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 8: count_launch(); launch_pdl(csc_back_kernel<V, 8, MODE>, blocks, kSpmvThreads, s, cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 16: count_launch(); launch_pdl(csc_back_kernel<V, 16, MODE>, blocks, kSpmvThreads, s, cp, ri, val, r, n, inv_n, ics, x, xs); break;
    default: count_launch(); launch_pdl(csc_back_kernel<V, 32, MODE>, blocks, kSpmvThreads, s, cp, ri, val, r, n, inv_n, ics, x, xs); break;
  }
}


template <typename V, int MODE, bool LL>
static void stream_fwd_launch(const mc_system *sys, const float *xs, const float *y, float *out, double *partials,
                              cudaStream_t s, const uint32_t *rmap = nullptr, const float *add = nullptr) {
  const unsigned nb = (unsigned)sys->n_csr_blocks;
  const uint32_t *rp = sys->row_ptr.as<uint32_t>(), *t = sys->csr_blocks.as<uint32_t>(), *ci = sys->col_idx.as<uint32_t>();
  const V *val = sys->csr_val.as<V>();
  count_launch();
  if (sys->warp_rows_fwd)
    stream_forward_kernel<V, true, MODE, LL><<<nb, kStreamThreads, 0, s>>>(rp, t, ci, val, xs, y, out, partials,
                                                                            rmap, add);
  else {
    const int R = chunk_rows_per_lane(sys->nnz, sys->n_rows, sys->n_rows);
    const unsigned g = (unsigned)div_up(sys->n_rows, (int64_t)kChunkThreads * R);
    const int64_t m = sys->n_rows;
    if (R == 1) launch_pdl(chunk_forward_kernel<1, V, MODE, LL>, g, kChunkThreads, s, rp, m, ci, val, xs, y, out, partials, rmap, add);
    else if (R == 2) launch_pdl(chunk_forward_kernel<2, V, MODE, LL>, g, kChunkThreads, s, rp, m, ci, val, xs, y, out, partials, rmap, add);
    else launch_pdl(chunk_forward_kernel<4, V, MODE, LL>, g, kChunkThreads, s, rp, m, ci, val, xs, y, out, partials, rmap, add);
  }
}

template <typename V, int MODE>
static void stream_back_launch(const mc_system *sys, const float *r, float *x, float *xs, cudaStream_t s) {
  const unsigned nb = (unsigned)sys->n_csc_blocks;
  const uint32_t *cp = sys->col_ptr.as<uint32_t>(), *t = sys->csc_blocks.as<uint32_t>(), *ri = sys->row_idx.as<uint32_t>();
  const V *val = sys->csc_val.as<V>();
  const float *inv_n = proj_scale(sys), *ics = proj_inv_norm(sys);
  count_launch();
  if (sys->warp_rows_bwd)
    stream_back_kernel<V, true, MODE><<<nb, kStreamThreads, 0, s>>>(cp, t, ri, val, r, inv_n, ics, x, xs);
  else {
    const int R = chunk_rows_per_lane(sys->nnz, sys->n_cols, sys->n_cols);
    const unsigned g = (unsigned)div_up(sys->n_cols, (int64_t)kChunkThreads * R);
    const int64_t n = sys->n_cols;
    if (R == 1) launch_pdl(chunk_back_kernel<1, V, MODE>, g, kChunkThreads, s, cp, n, ri, val, r, inv_n, ics, x, xs);
    else if (R == 2) launch_pdl(chunk_back_kernel<2, V, MODE>, g, kChunkThreads, s, cp, n, ri, val, r, inv_n, ics, x, xs);
    else launch_pdl(chunk_back_kernel<4, V, MODE>, g, kChunkThreads, s, cp, n, ri, val, r, inv_n, ics, x, xs);
  }
}

template <int MODE, bool LL>
static void fwd_dispatch(const mc_system *sys, const float *xs, const float *y, float *out, double *partials,
                         cudaStream_t s, const uint32_t *rmap = nullptr, const float *add = nullptr) {
  if (sys->n_csr_blocks > 0) {
    if (value_storage(sys->value_type) == 1) stream_fwd_launch<__half, MODE, LL>(sys, xs, y, out, partials, s, rmap, add);
    else if (value_storage(sys->value_type) == 2)
      stream_fwd_launch<__nv_bfloat16, MODE, LL>(sys, xs, y, out, partials, s, rmap, add);
    else stream_fwd_launch<float, MODE, LL>(sys, xs, y, out, partials, s, rmap, add);
    return;
  }
  const int g = sys->spmv_group_fwd;
  if (value_storage(sys->value_type) == 1) fwd_launch<__half, MODE, LL>(sys, g, xs, y, out, partials, s, rmap, add);
  else if (value_storage(sys->value_type) == 2) fwd_launch<__nv_bfloat16, MODE, LL>(sys, g, xs, y, out, partials, s, rmap, add);
  else fwd_launch<float, MODE, LL>(sys, g, xs, y, out, partials, s, rmap, add);
}

template <int MODE>
static void back_dispatch(const mc_system *sys, const float *r, float *x, float *xs, cudaStream_t s) {
  if (sys->n_csc_blocks > 0) {
    if (value_storage(sys->value_type) == 1) stream_back_launch<__half, MODE>(sys, r, x, xs, s);
    else if (value_storage(sys->value_type) == 2) stream_back_launch<__nv_bfloat16, MODE>(sys, r, x, xs, s);
    else stream_back_launch<float, MODE>(sys, r, x, xs, s);
    return;
  }
  const int g = sys->spmv_group_bwd;
  if (value_storage(sys->value_type) == 1) back_launch<__half, MODE>(sys, g, r, x, xs, s);
  else if (value_storage(sys->value_type) == 2) back_launch<__nv_bfloat16, MODE>(sys, g, r, x, xs, s);
  else back_launch<float, MODE>(sys, g, r, x, xs, s);
}

int forward_blocks(const mc_system *sys) {
  if (sys->n_csr_blocks > 0 && !sys->warp_rows_fwd)  // warp chunks
    return div_up(sys->n_rows, (int64_t)kChunkThreads * chunk_rows_per_lane(sys->nnz, sys->n_rows, sys->n_rows));
  if (sys->n_csr_blocks > 0) return (int)sys->n_csr_blocks;
  return div_up(sys->n_rows * sys->spmv_group_fwd, kSpmvThreads);
}

// Tiles for one pointer array.  Unless `force`, none (row-group kernels)
// when a segment is longer than half a tile or the mean segment is long;
// with `force` a segment longer than half a tile is an error.
static int stream_tiles(const DevBuf &ptr, int64_t n, int64_t nnz, DevBuf &tiles, int64_t &n_tiles, bool &warp,
                        cudaStream_t s, bool force = false) {
  n_tiles = 0;
  if (n <= 0 || nnz <= 0) return MC_OK;
  DevBuf mx;
  MCS_TRY(mx.alloc(sizeof(unsigned int), s));
  MCS_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned int), s));
  count_launch();
  max_segment_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(ptr.as<uint32_t>(), n, mx.as<unsigned int>());
  MCS_LAUNCHED();
  unsigned int longest = 0;
  MCS_CUDA(cudaMemcpyAsync(&longest, mx.p, sizeof(longest), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  if ((int64_t)longest * 2 > kStreamTile) {
    if (!force) return MC_OK;
    set_error("segment of %u entries is too long for a streaming tile", longest);
    return MC_EINVAL;
  }
  // tiles pay off for short segments; long ones stream better per row group
  if (!force && (double)nnz / (double)n >= 32.0) return MC_OK;
  const uint32_t step = (uint32_t)(kStreamTile - longest - 1);
  n_tiles = (nnz + n + step - 1) / step;
  MCS_TRY(tiles.alloc((size_t)(n_tiles + 1) * sizeof(uint32_t), s));
  count_launch();
  tile_bounds_kernel<<<grid_stride_blocks(n_tiles + 1), 256, 0, s>>>(ptr.as<uint32_t>(), n, step, n_tiles,
                                                                     tiles.as<uint32_t>());
  MCS_LAUNCHED();
  warp = (double)nnz / (double)n >= 16.0;
  return MC_OK;
}

// Forced projector layouts (mc_system_set_spmv_layout): 0 = streaming
// tiles (made now if the system has none), 1..32 = lanes per row group,
// -1 = keep.  On an error the system keeps its previous layout.
int set_spmv_layout(mc_system *sys, int fwd, int bwd, cudaStream_t s) {
  auto ok = [](int g) { return g == -1 || g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32; };
  if (!ok(fwd) || !ok(bwd)) {
    set_error("layouts must be -1 (keep), 0 (streaming tiles) or 1, 2, 4, 8, 16, 32 lanes; got %d, %d", fwd, bwd);
    return MC_EINVAL;
  }
  DevBuf ft, bt;
  int64_t nft = 0, nbt = 0;
  bool fw = sys->warp_rows_fwd, bw = sys->warp_rows_bwd;
  if (fwd == 0 && sys->n_csr_blocks == 0)
    MCS_TRY(stream_tiles(sys->row_ptr, sys->n_rows, sys->nnz, ft, nft, fw, s, true));
  if (bwd == 0 && sys->n_csc_blocks == 0)
    MCS_TRY(stream_tiles(sys->col_ptr, sys->n_cols, sys->nnz, bt, nbt, bw, s, true));
  if (fwd == 0 && sys->n_csr_blocks == 0) { sys->csr_blocks = std::move(ft); sys->n_csr_blocks = nft; sys->warp_rows_fwd = fw; }
  if (bwd == 0 && sys->n_csc_blocks == 0) { sys->csc_blocks = std::move(bt); sys->n_csc_blocks = nbt; sys->warp_rows_bwd = bw; }
  if (fwd > 0) { sys->n_csr_blocks = 0; sys->spmv_group_fwd = fwd; }
  if (bwd > 0) { sys->n_csc_blocks = 0; sys->spmv_group_bwd = bwd; }
  // the log-likelihood partials must cover the forward blocks of the layout
  const int fb = forward_blocks(sys);
  if ((size_t)fb * sizeof(double) > sys->partials.bytes) MCS_TRY(sys->partials.alloc((size_t)fb * sizeof(double), s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int make_stream_blocks(mc_system *sys, cudaStream_t s) {
  MCS_TRY(stream_tiles(sys->row_ptr, sys->n_rows, sys->nnz, sys->csr_blocks, sys->n_csr_blocks, sys->warp_rows_fwd, s));
  MCS_TRY(stream_tiles(sys->col_ptr, sys->n_cols, sys->nnz, sys->csc_blocks, sys->n_csc_blocks, sys->warp_rows_bwd, s));
  return MC_OK;
}

int project(const mc_system *sys, const float *x, float *q, cudaStream_t s) {
  if (sys->n_cols > 0) {
    count_launch(); prescale_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(x, proj_scale(sys), sys->xs.as<float>(),
                                                                     sys->n_cols);
  }
  if (sys->n_rows > 0) fwd_dispatch<0, false>(sys, sys->xs.as<float>(), nullptr, q, nullptr, s);
  MCS_LAUNCHED();
  return MC_OK;
}

// r = y / (A x), 0 where A x = 0 (the ratio of Eq. (MLEM))
int project_ratio(const mc_system *sys, const float *x, const float *y, float *r, cudaStream_t s) {
  if (sys->n_cols > 0) {
    count_launch();
    prescale_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(x, proj_scale(sys), sys->xs.as<float>(),
                                                                     sys->n_cols);
  }
  if (sys->n_rows > 0) fwd_dispatch<1, false>(sys, sys->xs.as<float>(), y, r, nullptr, s);
  MCS_LAUNCHED();
  return MC_OK;
}

// L(x) = sum_j y_j ln q_j - q_j (FP64), q = A x, into *value (device)
int loglik(const mc_system *sys, const float *x, const float *y, double *value, cudaStream_t s) {
  if (sys->n_cols > 0) {
    count_launch();
    prescale_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(x, proj_scale(sys), sys->xs.as<float>(),
                                                                     sys->n_cols);
  }
  if (sys->n_rows > 0) {
    fwd_dispatch<1, true>(sys, sys->xs.as<float>(), y, sys->r.as<float>(), sys->partials.as<double>(), s);
    count_launch();
    sum_partials_kernel<<<1, 1024, 0, s>>>(sys->partials.as<double>(), forward_blocks(sys), value);
  } else {
    MCS_CUDA(cudaMemsetAsync(value, 0, sizeof(double), s));
  }
  MCS_LAUNCHED();
  return MC_OK;
}

int backproject(const mc_system *sys, const float *r, float *b, cudaStream_t s) {
  if (sys->n_cols > 0) back_dispatch<0>(sys, r, b, nullptr, s);
  MCS_LAUNCHED();
  return MC_OK;
}

int sensitivity(const mc_system *sys, double *out, cudaStream_t s) {
  if (sys->n_cols > 0) {
    const uint32_t *nv = nullptr;
    const double *cs = proj_sens_terms(sys, &nv);
    count_launch(); sensitivity_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(cs, nv, sys->n_cols, out);
  }
  MCS_LAUNCHED();
  return MC_OK;
}

// FP64 sum of n floats (or doubles) in a fixed order: block partials over a
// fixed grid, then one block
template <typename T>
__global__ void partial_sums_kernel(const T *v, int64_t n, double *part) {
  __shared__ double s_tmp[32];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)v[i];
  const double t = block_sum_double(acc, s_tmp);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

int vector_sum(int64_t n, const float *v, double *out, cudaStream_t s) {
  const int nb = 256;
  DevBuf part;
  MCS_TRY(part.alloc(nb * sizeof(double), s));
  count_launch();
  partial_sums_kernel<float><<<nb, 256, 0, s>>>(v, n, part.as<double>());
  count_launch();
  sum_partials_kernel<<<1, 1024, 0, s>>>(part.as<double>(), nb, out);
  MCS_LAUNCHED();
  return MC_OK;
}

// x_v = sum_y / (sum of sens) where sens_v > 0, else 0 (the uniform start
// image of ML-EM from a sensitivity summed over several systems)
__global__ void start_fill_kernel(const double *total, double sum_y, const double *sens, int64_t n, float *x) {
  const double ts = *total;
  const float x0 = ts > 0.0 ? (float)(sum_y / ts) : 0.0f;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    x[v] = sens[v] > 0.0 ? x0 : 0.0f;
}

int mlem_start(int64_t n, const double *sens, double sum_y, float *x, cudaStream_t s) {
  const int nb = 256;
  DevBuf part;
  MCS_TRY(part.alloc((nb + 1) * sizeof(double), s));
  count_launch();
  partial_sums_kernel<double><<<nb, 256, 0, s>>>(sens, n, part.as<double>());
  count_launch();
  sum_partials_kernel<<<1, 1024, 0, s>>>(part.as<double>(), nb, part.as<double>() + nb);
  if (n > 0) {
    count_launch();
    start_fill_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(part.as<double>() + nb, sum_y, sens, n, x);
  }
  MCS_LAUNCHED();
  return MC_OK;
}

int mlem_init(mc_system *sys, const float *y, float *x, cudaStream_t s) {
  const int nb = 256;
  DevBuf part;
  MCS_TRY(part.alloc((2 * nb + 1) * sizeof(double), s));
  double *py = part.as<double>(), *ps = py + nb, *x0 = py + 2 * nb;
  const uint32_t *nv = nullptr;
  const double *cs = proj_sens_terms(sys, &nv);
  count_launch();
  init_sums_kernel<<<nb, 256, 0, s>>>(y, sys->n_rows, cs, nv, sys->n_cols, py, ps);
  count_launch();
  init_total_kernel<<<1, 256, 0, s>>>(py, ps, nb, x0);
  MCS_LAUNCHED();
  if (sys->n_cols > 0) {
    count_launch();
    init_fill_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(x0, cs, proj_scale(sys), sys->n_cols, x,
                                                                     sys->xs.as<float>());
  }
  MCS_LAUNCHED();
  return MC_OK;
}

// Ordered-subset EM sweeps: for each subset s, forward with fwd[s] (ratio
// with the additive term and the subset's row map), back-projection and
// update with back[s] (its column sums; voxels the subset does not see keep
// their value).  fwd and back may differ (dual
// matrix, Eq. (DMOS)); one subset with fwd = back is ML-EM.
int osem_run(mc_system *const *fwd, mc_system *const *back, int n_sub, const float *y, const float *add, float *x,
             int n_iter, cudaStream_t s) {
  for (int it = 0; it < n_iter; ++it) {
    for (int k = 0; k < n_sub; ++k) {
      mc_system *f = fwd[k], *b = back[k];
      const int64_t n = f->n_cols;
      if (n > 0) {
        count_launch();
        prescale_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x, proj_scale(f), f->xs.as<float>(), n);
      }
      if (f->n_rows > 0)
        fwd_dispatch<2, false>(f, f->xs.as<float>(), y, f->r.as<float>(), nullptr, s,
                               f->row_map.p ? f->row_map.as<uint32_t>() : nullptr, add);
      if (n > 0) back_dispatch<3>(b, f->r.as<float>(), x, b->xs.as<float>(), s);
      MCS_LAUNCHED();
    }
  }
  return MC_OK;
}

int mlem_run(mc_system *sys, const float *y, float *x, int n_iter, bool want_ll, cudaStream_t s) {
  const int64_t m = sys->n_rows, n = sys->n_cols;
  if (n > 0) {
    count_launch(); prescale_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x, proj_scale(sys), sys->xs.as<float>(), n);
  }
  MCS_LAUNCHED();
  const int fb = forward_blocks(sys);
  for (int k = 0; k < n_iter; ++k) {
    if (m > 0) {
      if (want_ll) {
        fwd_dispatch<1, true>(sys, sys->xs.as<float>(), y, sys->r.as<float>(), sys->partials.as<double>(), s);
        count_launch(); sum_partials_kernel<<<1, 1024, 0, s>>>(sys->partials.as<double>(), fb, sys->ll.as<double>() + k);
      } else {
        fwd_dispatch<1, false>(sys, sys->xs.as<float>(), y, sys->r.as<float>(), nullptr, s);
      }
    } else if (want_ll) {
      MCS_CUDA(cudaMemsetAsync(sys->ll.as<double>() + k, 0, sizeof(double), s));
    }
    if (n > 0) back_dispatch<1>(sys, sys->r.as<float>(), x, sys->xs.as<float>(), s);
    MCS_LAUNCHED();
  }
  return MC_OK;
}

}  // namespace mcs

// ---------------------------------------------------------------------------
// ML-EM without any device allocation
// ---------------------------------------------------------------------------
// Scratch of mlem_iterate_noalloc lives in this file-scope device array: one
// copy per GPU that loads the library, held until the process exits.  It
// holds the ratio vector r (M floats), the scaled image xs (N floats), the
// per-block log-likelihood partials and the per-iteration log-likelihoods.
namespace mcs {
constexpr int64_t kNoAllocRows = int64_t(1) << 21;   // largest M
constexpr int64_t kNoAllocCols = int64_t(1) << 21;   // largest N
constexpr int64_t kNoAllocPartials = kNoAllocRows * 32 / kSpmvThreads;  // forward blocks at 32 lanes/row
constexpr int64_t kNoAllocIters = 4096;              // log-likelihood values per call
constexpr size_t kNoAllocOffR = 0;
constexpr size_t kNoAllocOffXs = kNoAllocOffR + sizeof(float) * kNoAllocRows;
constexpr size_t kNoAllocOffPart = kNoAllocOffXs + sizeof(float) * kNoAllocCols;
constexpr size_t kNoAllocOffLl = kNoAllocOffPart + sizeof(double) * kNoAllocPartials;
constexpr size_t kNoAllocBytes = kNoAllocOffLl + sizeof(double) * kNoAllocIters;  // ~18 MiB

static __device__ __align__(256) unsigned char g_mlem_scratch[kNoAllocBytes];

// Device address of g_mlem_scratch on the current device (host code may not
// use the symbol itself: on the host it names a stand-in, not device memory).
static int noalloc_scratch(unsigned char **out) {
  static std::mutex mu;
  static void *addr[256] = {};
  int dev = 0;
  MCS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) { set_error("device ordinal %d out of range", dev); return MC_EINVAL; }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    MCS_CUDA(cudaGetSymbolAddress(&p, g_mlem_scratch));
    addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(addr[dev]);
  return MC_OK;
}
}  // namespace mcs

extern "C" int mlem_iterate_noalloc(const mc_system *sys, const float *y_dev, float *x_dev, int32_t n_iter,
                                    double *loglik_host, void *stream) {
  using namespace mcs;
  clear_error();
  if (!sys || !y_dev || !x_dev) { set_error("NULL argument"); return MC_EINVAL; }
  if (n_iter < 0) { set_error("n_iter must be >= 0"); return MC_EINVAL; }
  if (sys->n_rows > kNoAllocRows || sys->n_cols > kNoAllocCols) {
    set_error("mlem_iterate_noalloc: system of %lld rows x %lld columns exceeds the static scratch limit of "
              "%lld rows x %lld columns; use mlem_iterate",
              (long long)sys->n_rows, (long long)sys->n_cols, (long long)kNoAllocRows, (long long)kNoAllocCols);
    return MC_EINVAL;
  }
  const bool want = loglik_host != nullptr && n_iter > 0;
  if (want && n_iter > kNoAllocIters) {
    set_error("mlem_iterate_noalloc: at most %lld log-likelihood values per call", (long long)kNoAllocIters);
    return MC_EINVAL;
  }
  const int fb = forward_blocks(sys);
  if (fb > kNoAllocPartials) {
    set_error("mlem_iterate_noalloc: %d forward blocks exceed the static limit %lld", fb, (long long)kNoAllocPartials);
    return MC_EINVAL;
  }
  // the scratch array used is the current device's: it must be the device
  // that holds the system's matrix and work vectors
  int dev = -1;
  MCS_CUDA(cudaGetDevice(&dev));
  if (dev != sys->device) {
    set_error("mlem_iterate_noalloc: the current device is %d but the system was built on device %d; make the "
              "system's device current first",
              dev, sys->device);
    return MC_EINVAL;
  }
  unsigned char *base = nullptr;
  MCS_TRY(noalloc_scratch(&base));
  float *r = reinterpret_cast<float *>(base + kNoAllocOffR);
  float *xs = reinterpret_cast<float *>(base + kNoAllocOffXs);
  double *partials = reinterpret_cast<double *>(base + kNoAllocOffPart);
  double *ll = reinterpret_cast<double *>(base + kNoAllocOffLl);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t m = sys->n_rows, n = sys->n_cols;
  // every scratch element is written before it is read: nothing to clear
  if (n > 0) {
    count_launch();
    prescale_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x_dev, proj_scale(sys), xs, n);
  }
  MCS_LAUNCHED();
  for (int k = 0; k < n_iter; ++k) {
    if (m > 0) {
      if (want) {
        fwd_dispatch<1, true>(sys, xs, y_dev, r, partials, s);
        count_launch();
        sum_partials_kernel<<<1, 1024, 0, s>>>(partials, fb, ll + k);
      } else {
        fwd_dispatch<1, false>(sys, xs, y_dev, r, nullptr, s);
      }
    } else if (want) {
      MCS_CUDA(cudaMemsetAsync(ll + k, 0, sizeof(double), s));
    }
    if (n > 0) back_dispatch<1>(sys, r, x_dev, xs, s);
    MCS_LAUNCHED();
  }
  if (want) {
    MCS_CUDA(cudaMemcpyAsync(loglik_host, ll, (size_t)n_iter * sizeof(double), cudaMemcpyDeviceToHost, s));
    MCS_CUDA(cudaStreamSynchronize(s));
  }
  return MC_OK;
}

// ---------------------------------------------------------------------------
// double-precision projectors, quadratic prior, preconditioned gradient step
// (the differentiable / penalised forms built on Eq. (IMC) and the Poisson
// likelihood of Sec. 5.1)
// ---------------------------------------------------------------------------
namespace mcs {

// q_j = sum_v C_jv x_v / n_v, one thread per row, double accumulation
// entry k as a double: the count, or (weighted systems) the fixed-point
// weight sum
__device__ __forceinline__ double entry_f64(const uint32_t *cnt, const uint64_t *wq, uint32_t k) {
  return wq ? (double)wq[k] * (1.0 / kFdScale) : (double)cnt[k];
}

__global__ void forward_f64_kernel(const uint32_t *row_ptr, const uint32_t *col, const uint32_t *cnt,
                                   const uint64_t *wq, const uint32_t *n_v, const double *x, int64_t m, double *q) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (uint32_t k = row_ptr[j]; k < row_ptr[j + 1]; ++k) {
      const uint32_t v = col[k];
      acc += entry_f64(cnt, wq, k) * (x[v] / (double)n_v[v]);
    }
    q[j] = acc;
  }
}

// b_v = (1/n_v) sum_j C_jv r_j
__global__ void back_f64_kernel(const uint32_t *col_ptr, const uint32_t *row, const uint32_t *cnt,
                                const uint64_t *wq, const uint32_t *n_v, const double *r, int64_t n, double *b) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (uint32_t k = col_ptr[v]; k < col_ptr[v + 1]; ++k) acc += entry_f64(cnt, wq, k) * r[row[k]];
    b[v] = n_v[v] ? acc / (double)n_v[v] : 0.0;
  }
}

// Quadratic 6-neighbour prior R(x) = beta/2 sum over neighbour pairs (x_v - x_w)^2
// (each pair once); grad_v = beta sum over the neighbours w of v (x_v - x_w).
template <typename T>
__global__ void prior_kernel(int nx, int ny, int nz, double beta, const T *x, T *grad, double *partials) {
  __shared__ double s_tmp[32];
  const int64_t n = (int64_t)nx * ny * nz;
  double val = 0.0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((int64_t)nx * ny));
    const double xv = (double)x[v];
    double g = 0.0;
    if (i > 0) g += xv - (double)x[v - 1];
    if (i < nx - 1) { const double d = xv - (double)x[v + 1]; g += d; val += d * d; }
    if (j > 0) g += xv - (double)x[v - nx];
    if (j < ny - 1) { const double d = xv - (double)x[v + nx]; g += d; val += d * d; }
    if (k > 0) g += xv - (double)x[v - (int64_t)nx * ny];
    if (k < nz - 1) { const double d = xv - (double)x[v + (int64_t)nx * ny]; g += d; val += d * d; }
    if (grad) grad[v] = (T)(beta * g);
  }
  if (partials) {
    const double t = block_sum_double(0.5 * beta * val, s_tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// x_v <- max(0, x_v - alpha (x_v / s_v) (s_v - bp_v + gp_v)): gradient descent on
// sum_j (q_j - y_j ln q_j) + R(x) with the EM preconditioner x / s; alpha = 1
// and no prior is one ML-EM update.  Voxels with s_v = 0 are set to 0.
__global__ void pgd_step_kernel(int64_t n, double alpha, const double *sens, const float *bp, const float *gp,
                                float *x) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const double s = sens[v];
    if (!(s > 0.0)) { x[v] = 0.0f; continue; }
    const double grad = s - (double)bp[v] + (gp ? (double)gp[v] : 0.0);
    const double xn = (double)x[v] - alpha * ((double)x[v] / s) * grad;
    x[v] = (float)(xn > 0.0 ? xn : 0.0);
  }
}

int project_f64(const mc_system *sys, const double *x, double *q, cudaStream_t s) {
  if (sys->n_rows > 0) {
    count_launch();
    forward_f64_kernel<<<grid_stride_blocks(sys->n_rows), 256, 0, s>>>(
        sys->row_ptr.as<uint32_t>(), sys->col_idx.as<uint32_t>(), sys->csr_cnt.as<uint32_t>(),
        sys->weighted ? sys->csr_wq.as<uint64_t>() : nullptr, sys->n_v.as<uint32_t>(), x, sys->n_rows, q);
  }
  MCS_LAUNCHED();
  return MC_OK;
}

int backproject_f64(const mc_system *sys, const double *r, double *b, cudaStream_t s) {
  if (sys->n_cols > 0) {
    count_launch();
    back_f64_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(
        sys->col_ptr.as<uint32_t>(), sys->row_idx.as<uint32_t>(), sys->csc_cnt.as<uint32_t>(),
        sys->weighted ? sys->csc_wq.as<uint64_t>() : nullptr, sys->n_v.as<uint32_t>(), r, sys->n_cols, b);
  }
  MCS_LAUNCHED();
  return MC_OK;
}

template <typename T>
int prior_quadratic(int nx, int ny, int nz, double beta, const T *x, T *grad, double *value, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int nb = grid_stride_blocks(n);
  DevBuf part;
  if (value) MCS_TRY(part.alloc((size_t)nb * sizeof(double), s));
  count_launch();
  prior_kernel<T><<<nb, 256, 0, s>>>(nx, ny, nz, beta, x, grad, value ? part.as<double>() : nullptr);
  MCS_LAUNCHED();
  if (value) {
    count_launch();
    sum_partials_kernel<<<1, 1024, 0, s>>>(part.as<double>(), nb, value);
    MCS_LAUNCHED();
  }
  return MC_OK;
}
template int prior_quadratic<float>(int, int, int, double, const float *, float *, double *, cudaStream_t);
template int prior_quadratic<double>(int, int, int, double, const double *, double *, double *, cudaStream_t);

int pgd_step(int64_t n, double alpha, const double *sens, const float *bp, const float *gp, float *x, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    pgd_step_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(n, alpha, sens, bp, gp, x);
  }
  MCS_LAUNCHED();
  return MC_OK;
}

}  // namespace mcs

// ---------------------------------------------------------------------------
// batched ML-EM over many systems (serving many acquisitions at once)
// ---------------------------------------------------------------------------
// Each iteration is one forward launch over the concatenated CSR work units
// of all systems and one back-projection launch over their CSC units; a
// block finds its system by binary search in the prefix of unit counts.  A
// unit is 256 R consecutive rows (columns) as eight warp chunks, or, for a
// system whose rows (columns) average 16 or more entries, one tile with a
// warp per row (column).  The
// whole reconstruction (start images, n_iter iterations, write-back of the
// images) is captured once in a CUDA graph and replayed.
//
// Serving systems are built from few histories, so most of their rows and
// columns are empty.  The batch renumbers each system onto its non-empty
// rows and columns only: compacted pointers, row/column indices relabelled
// to compacted positions, and per-system compacted vectors (y, ratio, image,
// scaled image, 1/S, 1/n_v).  An empty row's ratio is never read (no column
// refers to it), and an empty column has S_v = 0, so the start image sets it
// to 0 and the update keeps it there: the iterates are those of the full
// system.  An iteration then streams bytes in proportion to the non-zeros,
// and the gathered vectors (4 bytes per non-empty column or row) stay in L2.
namespace mcs {

struct BatchSys {
  // compacted CSR: segment j is row row_id[j], entries [row_ptr[j],
  // row_ptr[j + 1]) with column indices in compacted column numbering;
  // tiles only where warp_fwd (warp_bwd) is set
  const uint32_t *row_ptr, *row_id, *csr_tiles, *col_idx;
  // compacted CSC: segment j is column col_id[j]; row indices compacted
  const uint32_t *col_ptr, *col_id, *csc_tiles, *row_idx;
  const float *csr_val, *csc_val;
  const float *y;            // measured data, all n_rows rows
  float *x;                  // image, all n_cols voxels
  float *y_c, *r_c;          // per non-empty row: data, ratio y / (A x)
  float *x_c, *xs_c;         // per non-empty column: image, image / n_v
  const float *ics_c, *invn_c;  // per non-empty column: 1 / S_v, 1 / n_v
  int64_t n_rows, n_cols, m_c, n_c;
  int warp_fwd, warp_bwd;  // tiles with a warp per segment, else warp chunks
  int rpl_fwd, rpl_bwd;    // warp chunks: segments per lane
};

__device__ __forceinline__ int batch_find(const uint64_t *off, int n, uint64_t i) {
  int lo = 0, hi = n - 1;  // largest k with off[k] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The block's system descriptor for global tile t is copied to shared
// memory once, so that stores through its output pointers cannot force
// reloads of the others.
__device__ __forceinline__ const BatchSys &batch_desc(const BatchSys *systems, const uint64_t *off, int n_sys,
                                                      BatchSys *s_desc, uint64_t t, uint32_t &tile) {
  const int k = batch_find(off, n_sys, t);
  if (threadIdx.x == 0) *s_desc = systems[k];
  tile = (uint32_t)(t - off[k]);
  __syncthreads();
  return *s_desc;
}

// batch epilogues on compacted vectors: r_c = y_c / q (0 where q = 0);
// x_c <- x_c t / S, xs_c = x_c / n_v
struct BatchFwdOut {
  using Pre = float;
  const float *__restrict__ y;
  float *__restrict__ r;
  __device__ __forceinline__ float load(uint32_t j) const { return y[j]; }
  __device__ __forceinline__ void store(uint32_t j, float acc, float yv, bool) const { r[j] = acc > 0.0f ? yv / acc : 0.0f; }
};

// Unit u of a warp-chunk system: its block's warps take the chunks of
// segments [256 R u, 256 R (u + 1)).
template <typename Out>
__device__ __forceinline__ void batch_chunks(const uint32_t *__restrict__ ptr, int64_t n_seg,
                                             const uint32_t *__restrict__ idx, const float *__restrict__ val,
                                             const float *__restrict__ vec, float *s_prod, Out &o, uint32_t u,
                                             int R) {
  float *s_w = s_prod + (threadIdx.x >> 5) * kChunkWindow;
  const int64_t j0 = ((int64_t)u * kStreamThreads + (threadIdx.x & ~31u)) * R;
  if (R == 1) chunk_segments<1, float>(ptr, n_seg, idx, val, vec, s_w, o, j0);
  else if (R == 2) chunk_segments<2, float>(ptr, n_seg, idx, val, vec, s_w, o, j0);
  else chunk_segments<4, float>(ptr, n_seg, idx, val, vec, s_w, o, j0);
}

// One forward (ratio) tile and one back-projection (EM update) tile of the
// batch, by global tile index t
__device__ __forceinline__ void batch_forward_tile(const BatchSys *__restrict__ systems,
                                                   const uint64_t *__restrict__ tile_off, int n_sys, uint64_t t,
                                                   float *s_prod, BatchSys *s_desc) {
  uint32_t tile;
  const BatchSys &S = batch_desc(systems, tile_off, n_sys, s_desc, t, tile);
  const uint32_t *__restrict__ ptr = S.row_ptr;
  BatchFwdOut o{S.y_c, S.r_c};
  if (!S.warp_fwd) {  // warp chunks over rows [256 R u, 256 R (u + 1))
    batch_chunks(ptr, S.m_c, S.col_idx, S.csr_val, S.xs_c, s_prod, o, tile, S.rpl_fwd);
    return;
  }
  const uint32_t j0 = S.csr_tiles[tile], j1 = S.csr_tiles[tile + 1];
  const uint32_t p0 = ptr[j0];
  stream_products<float>(p0, ptr[j1] - p0, S.col_idx, S.csr_val, S.xs_c, s_prod);
  __syncthreads();
  stream_segments<true>(ptr, j0, j1, p0, s_prod, o);
}

__device__ __forceinline__ void batch_back_tile(const BatchSys *__restrict__ systems,
                                                const uint64_t *__restrict__ tile_off, int n_sys, uint64_t t,
                                                float *s_prod, BatchSys *s_desc) {
  uint32_t tile;
  const BatchSys &S = batch_desc(systems, tile_off, n_sys, s_desc, t, tile);
  const uint32_t *__restrict__ ptr = S.col_ptr;
  BackOut<1> o{S.invn_c, S.ics_c, S.x_c, S.xs_c};
  if (!S.warp_bwd) {  // warp chunks over columns [256 R u, 256 R (u + 1))
    batch_chunks(ptr, S.n_c, S.row_idx, S.csc_val, S.r_c, s_prod, o, tile, S.rpl_bwd);
    return;
  }
  const uint32_t j0 = S.csc_tiles[tile], j1 = S.csc_tiles[tile + 1];
  const uint32_t p0 = ptr[j0];
  stream_products<float>(p0, ptr[j1] - p0, S.row_idx, S.csc_val, S.r_c, s_prod);
  __syncthreads();
  stream_segments<true>(ptr, j0, j1, p0, s_prod, o);
}

__global__ void __launch_bounds__(kStreamThreads) batch_forward_kernel(const BatchSys *__restrict__ systems,
                                                                    const uint64_t *__restrict__ tile_off,
                                                                    int n_sys) {
  __shared__ float s_prod[kStreamTile];
  __shared__ BatchSys s_desc;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  batch_forward_tile(systems, tile_off, n_sys, blockIdx.x, s_prod, &s_desc);
}

__global__ void __launch_bounds__(kStreamThreads) batch_back_kernel(const BatchSys *__restrict__ systems,
                                                                 const uint64_t *__restrict__ tile_off, int n_sys) {
  __shared__ float s_prod[kStreamTile];
  __shared__ BatchSys s_desc;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  batch_back_tile(systems, tile_off, n_sys, blockIdx.x, s_prod, &s_desc);
}

// All n_iter iterations of every system in one cooperative launch: the
// blocks stay resident, take the forward tiles in a grid-stride loop, meet
// at a grid-wide barrier, take the back-projection tiles, and meet again
// (the barrier the separate launches give).  Launched only through
// cudaLaunchCooperativeKernel with every block resident.
__global__ void __launch_bounds__(kStreamThreads) batch_persistent_kernel(const BatchSys *__restrict__ systems,
                                                                       const uint64_t *__restrict__ tile_fwd,
                                                                       uint64_t n_fwd,
                                                                       const uint64_t *__restrict__ tile_bwd,
                                                                       uint64_t n_bwd, int n_sys, int n_iter) {
  __shared__ float s_prod[kStreamTile];
  __shared__ BatchSys s_desc;
  cooperative_groups::grid_group grid = cooperative_groups::this_grid();
  for (int it = 0; it < n_iter; ++it) {
    for (uint64_t t = blockIdx.x; t < n_fwd; t += gridDim.x) {
      batch_forward_tile(systems, tile_fwd, n_sys, t, s_prod, &s_desc);
      __syncthreads();  // s_prod and s_desc are reused by the next tile
    }
    grid.sync();
    for (uint64_t t = blockIdx.x; t < n_bwd; t += gridDim.x) {
      batch_back_tile(systems, tile_bwd, n_sys, t, s_prod, &s_desc);
      __syncthreads();
    }
    grid.sync();
  }
}

// Non-empty segments of a pointer array: flags (1 per non-empty segment,
// 0 at index n), then after an exclusive scan of the flags each non-empty
// segment i lands at pos[i] with its id and start; cptr[count] = ptr[n].
__global__ void segment_flags_kernel(const uint32_t *ptr, int64_t n, uint32_t *flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = i < n && ptr[i + 1] > ptr[i] ? 1u : 0u;
}

__global__ void segment_compact_kernel(const uint32_t *ptr, int64_t n, const uint32_t *flags, const uint32_t *pos,
                                       uint32_t *id, uint32_t *cptr) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    if (i == n) cptr[pos[n]] = ptr[n];
    else if (flags[i]) { id[pos[i]] = (uint32_t)i; cptr[pos[i]] = ptr[i]; }
  }
}

// out[e] = pos[idx[e]]: entry indices in compacted numbering
__global__ void relabel_kernel(const uint32_t *idx, int64_t nnz, const uint32_t *pos, uint32_t *out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = pos[idx[e]];
}

__global__ void gather_f32_kernel(const float *src, const uint32_t *id, int64_t n, float *dst) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = src[id[j]];
}

// Start images: x0_k = sum(y_k) / sum(s_k).  The sensitivity totals are a
// property of the systems and are summed once when the batch is made; sum(y)
// runs over kInitChunks slices per system, then in a fixed order.  Every
// per-system kernel below is a row of kInitChunks blocks per system.
constexpr int kInitChunks = 64;
__global__ void batch_sens_sums_kernel(const double *const *colsum, const uint32_t *const *n_v, const int64_t *n_cols,
                                       double *part) {
  __shared__ double s_tmp[32];
  const int k = blockIdx.x / kInitChunks, c = blockIdx.x % kInitChunks;
  const double *cs = colsum[k];
  const uint32_t *nv = n_v[k];
  double as = 0.0;
  for (int64_t v = (int64_t)c * blockDim.x + threadIdx.x; v < n_cols[k]; v += (int64_t)kInitChunks * blockDim.x)
    if (nv[v]) as += cs[v] / (double)nv[v];
  const double ts = block_sum_double(as, s_tmp);
  if (threadIdx.x == 0) part[blockIdx.x] = ts;
}

__device__ __forceinline__ const BatchSys &batch_row_desc(const BatchSys *systems, BatchSys *s_desc, int &k, int &c) {
  k = blockIdx.x / kInitChunks;
  c = blockIdx.x % kInitChunks;
  if (threadIdx.x == 0) *s_desc = systems[k];
  __syncthreads();
  return *s_desc;
}

// partial sums of y, and x = 0 over the whole image (the non-empty columns
// are written back at the end)
__global__ void batch_init_sums_kernel(const BatchSys *systems, double *part) {
  __shared__ double s_tmp[32];
  __shared__ BatchSys s_desc;
  int k, c;
  const BatchSys &S = batch_row_desc(systems, &s_desc, k, c);
  const float *__restrict__ y = S.y;
  float *__restrict__ x = S.x;
  const int64_t stride = (int64_t)kInitChunks * blockDim.x, first = (int64_t)c * blockDim.x + threadIdx.x;
  double ay = 0.0;
  for (int64_t i = first; i < S.n_rows; i += stride) ay += (double)y[i];
  for (int64_t v = first; v < S.n_cols; v += stride) x[v] = 0.0f;
  const double ty = block_sum_double(ay, s_tmp);
  if (threadIdx.x == 0) part[blockIdx.x] = ty;
}

// x0[k] = (sum of part_y over k's chunks) / (sum of part_s over k's chunks)
__global__ void batch_init_total_kernel(const double *part_y, const double *part_s, int n_sys, double *x0) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_sys; k += gridDim.x * blockDim.x) {
    double sy = 0.0, ss = 0.0;
    for (int c = 0; c < kInitChunks; ++c) {
      sy += part_y[k * kInitChunks + c];
      ss += part_s[k * kInitChunks + c];
    }
    x0[k] = ss > 0.0 ? sy / ss : 0.0;
  }
}

// compacted data y_c, start image x_c = x0 (every compacted column has
// S > 0), xs_c = x_c / n_v
__global__ void batch_init_fill_kernel(const BatchSys *systems, const double *x0) {
  __shared__ BatchSys s_desc;
  int k, c;
  const BatchSys &S = batch_row_desc(systems, &s_desc, k, c);
  const int64_t stride = (int64_t)kInitChunks * blockDim.x, first = (int64_t)c * blockDim.x + threadIdx.x;
  const float x0k = (float)x0[k];
  for (int64_t j = first; j < S.m_c; j += stride) S.y_c[j] = S.y[S.row_id[j]];
  for (int64_t j = first; j < S.n_c; j += stride) {
    S.x_c[j] = x0k;
    S.xs_c[j] = x0k * S.invn_c[j];
  }
}

// image write-back: x[col_id[j]] = x_c[j]
__global__ void batch_scatter_kernel(const BatchSys *systems) {
  __shared__ BatchSys s_desc;
  int k, c;
  const BatchSys &S = batch_row_desc(systems, &s_desc, k, c);
  const int64_t stride = (int64_t)kInitChunks * blockDim.x, first = (int64_t)c * blockDim.x + threadIdx.x;
  for (int64_t j = first; j < S.n_c; j += stride) S.x[S.col_id[j]] = S.x_c[j];
}

}  // namespace mcs

// Per system the batch owns kBatchBufs device buffers (see batch_create).
constexpr int kBatchBufs = 14;

struct mc_batch {
  int n = 0;
  mcs::DevBuf systems, tile_fwd, tile_bwd, x0, part_y, part_s;
  std::vector<mcs::DevBuf> owned;  // kBatchBufs per system
  uint64_t n_tiles_fwd = 0, n_tiles_bwd = 0;
  cudaGraphExec_t exec = nullptr;
  int exec_iters = -1;
  ~mc_batch() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

namespace mcs {

// The non-empty segments of (ptr, n): their ids, compacted pointers, stream
// tiles (`warp` set, when segments average 16 or more entries; warp-chunk
// units are set by batch_create), and `relabel_out` = `relabel_in` (nnz
// indices into this numbering, from the other orientation) in compacted
// numbering.
// `scratch` holds 2 (n + 1) words.
static int batch_segments(const uint32_t *ptr, int64_t n, int64_t nnz, const uint32_t *relabel_in, uint32_t *scratch,
                          DevBuf &id, DevBuf &cptr, DevBuf &tiles, DevBuf &relabel_out, int64_t &count, int64_t &n_tiles,
                          int &warp, cudaStream_t s) {
  uint32_t *flags = scratch, *pos = scratch + (n + 1);
  count_launch();
  segment_flags_kernel<<<grid_stride_blocks(n + 1), 256, 0, s>>>(ptr, n, flags);
  MCS_LAUNCHED();
  MCS_TRY(exclusive_scan_u32(flags, pos, n + 1, s));
  uint32_t cnt = 0;
  MCS_CUDA(cudaMemcpyAsync(&cnt, pos + n, sizeof(cnt), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  count = cnt;
  MCS_TRY(id.alloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(uint32_t), s));
  MCS_TRY(cptr.alloc((size_t)(cnt + 1) * sizeof(uint32_t), s));
  MCS_TRY(relabel_out.alloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(uint32_t), s));
  count_launch();
  segment_compact_kernel<<<grid_stride_blocks(n + 1), 256, 0, s>>>(ptr, n, flags, pos, id.as<uint32_t>(),
                                                                    cptr.as<uint32_t>());
  MCS_LAUNCHED();
  if (nnz > 0) {
    count_launch();
    relabel_kernel<<<grid_stride_blocks(nnz), 256, 0, s>>>(relabel_in, nnz, pos, relabel_out.as<uint32_t>());
    MCS_LAUNCHED();
  }
  n_tiles = 0;
  warp = 0;
  if (cnt == 0) return MC_OK;
  if ((double)nnz / (double)cnt < 16.0) return MC_OK;  // warp chunks: units set by batch_create
  bool w = false;
  MCS_TRY(stream_tiles(cptr, cnt, nnz, tiles, n_tiles, w, s, true));
  warp = 1;
  return MC_OK;
}

// Per system k the batch owns, in owned[k * kBatchBufs + i]:
//   0 row ids  1 row pointers  2 CSR tiles  3 column indices (compacted)
//   4 col ids  5 col pointers  6 CSC tiles  7 row indices (compacted)
//   8 y_c  9 r_c  10 x_c  11 xs_c  12 1/S (compacted)  13 1/n_v (compacted)
int batch_create(mc_system *const *sys, int n, const float *const *y, float *const *x, mc_batch **out) {
  std::vector<BatchSys> hs(n);
  std::vector<uint64_t> tf(n + 1, 0), tb(n + 1, 0);
  std::vector<const double *> h_colsum(n);
  std::vector<const uint32_t *> h_nv(n);
  std::vector<int64_t> h_ncols(n);
  int64_t longest_vec = 1;
  for (int k = 0; k < n; ++k) {
    const mc_system *s = sys[k];
    if (!s || !y[k] || !x[k]) { set_error("batch entry %d: NULL system or vector", k); return MC_EINVAL; }
    // the batch builds its own work units over the non-empty rows and
    // columns (with tiles, an error if a row or column is longer than half
    // a tile)
    if (s->value_type != MC_VAL_F32 || s->row_map.p) {
      set_error("batch entry %d: needs a full (not ordered-subset) system with FP32 values", k);
      return MC_EINVAL;
    }
    longest_vec = std::max<int64_t>(longest_vec, std::max(s->n_rows, s->n_cols) + 1);
  }
  mc_batch *b = new (std::nothrow) mc_batch();
  if (!b) { set_error("out of host memory"); return MC_ENOMEM; }
  auto fail = [&](int rc) { delete b; return rc; };
  cudaStream_t s = nullptr;
  int rc;
  b->owned.resize((size_t)n * kBatchBufs);
  {
    DevBuf scratch;
    if ((rc = scratch.alloc((size_t)2 * longest_vec * sizeof(uint32_t), s))) return fail(rc);
    for (int k = 0; k < n; ++k) {
      const mc_system *m = sys[k];
      DevBuf *o = &b->owned[(size_t)k * kBatchBufs];
      int64_t nt_f = 0, nt_b = 0, m_c = 0, n_c = 0;
      BatchSys &d = hs[k];
      // rows: compacted CSR segments, and the CSC's row indices relabelled
      if ((rc = batch_segments(m->row_ptr.as<uint32_t>(), m->n_rows, m->nnz, m->row_idx.as<uint32_t>(),
                               scratch.as<uint32_t>(), o[0], o[1], o[2], o[7], m_c, nt_f, d.warp_fwd, s)) ||
          (rc = batch_segments(m->col_ptr.as<uint32_t>(), m->n_cols, m->nnz, m->col_idx.as<uint32_t>(),
                               scratch.as<uint32_t>(), o[4], o[5], o[6], o[3], n_c, nt_b, d.warp_bwd, s)))
        return fail(rc);
      for (int i = 8; i < 10; ++i)
        if ((rc = o[i].alloc((size_t)std::max<int64_t>(m_c, 1) * sizeof(float), s))) return fail(rc);
      for (int i = 10; i < 14; ++i)
        if ((rc = o[i].alloc((size_t)std::max<int64_t>(n_c, 1) * sizeof(float), s))) return fail(rc);
      if (n_c > 0) {
        count_launch();
        gather_f32_kernel<<<grid_stride_blocks(n_c), 256, 0, s>>>(m->inv_colsum.as<float>(), o[4].as<uint32_t>(), n_c,
                                                                  o[12].as<float>());
        count_launch();
        gather_f32_kernel<<<grid_stride_blocks(n_c), 256, 0, s>>>(m->inv_n.as<float>(), o[4].as<uint32_t>(), n_c,
                                                                  o[13].as<float>());
        if (cudaGetLastError() != cudaSuccess) { set_error("batch gather failed"); return fail(MC_ECUDA); }
      }
      d.row_id = o[0].as<uint32_t>(); d.row_ptr = o[1].as<uint32_t>(); d.csr_tiles = o[2].as<uint32_t>();
      d.col_idx = o[3].as<uint32_t>();
      d.col_id = o[4].as<uint32_t>(); d.col_ptr = o[5].as<uint32_t>(); d.csc_tiles = o[6].as<uint32_t>();
      d.row_idx = o[7].as<uint32_t>();
      d.csr_val = m->csr_val.as<float>(); d.csc_val = m->csc_val.as<float>();
      d.y = y[k]; d.x = x[k];
      d.y_c = o[8].as<float>(); d.r_c = o[9].as<float>(); d.x_c = o[10].as<float>(); d.xs_c = o[11].as<float>();
      d.ics_c = o[12].as<float>(); d.invn_c = o[13].as<float>();
      d.n_rows = m->n_rows; d.n_cols = m->n_cols; d.m_c = m_c; d.n_c = n_c;
      d.rpl_fwd = d.rpl_bwd = 1;
      tf[k + 1] = (uint64_t)nt_f;  // tiles; warp-chunk units below
      tb[k + 1] = (uint64_t)nt_b;
      h_colsum[k] = m->colsum.as<double>(); h_nv[k] = m->n_v.as<uint32_t>(); h_ncols[k] = m->n_cols;
    }
    MCS_CUDA(cudaStreamSynchronize(s));  // scratch is released on s after the last compaction
  }
  // warp-chunk systems: blocks of 256 R segments, R from the system's mean
  // segment length and the whole launch's segment count
  int64_t all_rows = 0, all_cols = 0;
  for (int k = 0; k < n; ++k) { all_rows += hs[k].m_c; all_cols += hs[k].n_c; }
  for (int k = 0; k < n; ++k) {
    BatchSys &d = hs[k];
    const int64_t nnz = sys[k]->nnz;
    if (!d.warp_fwd && d.m_c > 0) {
      d.rpl_fwd = chunk_rows_per_lane(nnz, d.m_c, all_rows);
      tf[k + 1] = (uint64_t)div_up(d.m_c, (int64_t)kStreamThreads * d.rpl_fwd);
    }
    if (!d.warp_bwd && d.n_c > 0) {
      d.rpl_bwd = chunk_rows_per_lane(nnz, d.n_c, all_cols);
      tb[k + 1] = (uint64_t)div_up(d.n_c, (int64_t)kStreamThreads * d.rpl_bwd);
    }
  }
  for (int k = 0; k < n; ++k) {
    tf[k + 1] += tf[k];
    tb[k + 1] += tb[k];
  }
  if (tf[n] >= (1ull << 31) || tb[n] >= (1ull << 31)) { set_error("too many tiles for one launch"); return fail(MC_EINVAL); }
  DevBuf d_cs, d_nv, d_nc;
  if ((rc = b->systems.alloc(n * sizeof(BatchSys), s)) || (rc = b->tile_fwd.alloc((n + 1) * 8, s)) ||
      (rc = b->tile_bwd.alloc((n + 1) * 8, s)) || (rc = b->x0.alloc(n * sizeof(double), s)) ||
      (rc = b->part_y.alloc((size_t)n * kInitChunks * sizeof(double), s)) ||
      (rc = b->part_s.alloc((size_t)n * kInitChunks * sizeof(double), s)) ||
      (rc = d_cs.alloc(n * sizeof(double *), s)) || (rc = d_nv.alloc(n * sizeof(uint32_t *), s)) ||
      (rc = d_nc.alloc(n * sizeof(int64_t), s)))
    return fail(rc);
  if (cudaMemcpyAsync(b->systems.p, hs.data(), n * sizeof(BatchSys), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->tile_fwd.p, tf.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b->tile_bwd.p, tb.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_cs.p, h_colsum.data(), n * sizeof(double *), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_nv.p, h_nv.data(), n * sizeof(uint32_t *), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(d_nc.p, h_ncols.data(), n * sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("batch upload failed");
    return fail(MC_ECUDA);
  }
  count_launch();
  batch_sens_sums_kernel<<<n * kInitChunks, 256, 0, s>>>(d_cs.as<const double *>(), d_nv.as<const uint32_t *>(),
                                                         d_nc.as<int64_t>(), b->part_s.as<double>());
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("batch sensitivity sums failed");
    return fail(MC_ECUDA);
  }
  b->n = n;
  b->n_tiles_fwd = tf[n];
  b->n_tiles_bwd = tb[n];
  *out = b;
  return MC_OK;
}

// Enqueue the whole batched reconstruction on s (used once for capture).
static int batch_enqueue(mc_batch *b, int n_iter, cudaStream_t s) {
  const BatchSys *sys = b->systems.as<BatchSys>();
  const unsigned rows = (unsigned)(b->n * kInitChunks);
  count_launch();
  batch_init_sums_kernel<<<rows, 256, 0, s>>>(sys, b->part_y.as<double>());
  count_launch();
  batch_init_total_kernel<<<div_up(b->n, 256), 256, 0, s>>>(b->part_y.as<double>(), b->part_s.as<double>(), b->n,
                                                            b->x0.as<double>());
  count_launch();
  batch_init_fill_kernel<<<rows, 256, 0, s>>>(sys, b->x0.as<double>());
  for (int it = 0; it < n_iter; ++it) {
    if (b->n_tiles_fwd) {
      count_launch();
      launch_pdl(batch_forward_kernel, (unsigned)b->n_tiles_fwd, kStreamThreads, s, sys, b->tile_fwd.as<uint64_t>(), b->n);
    }
    if (b->n_tiles_bwd) {
      count_launch();
      launch_pdl(batch_back_kernel, (unsigned)b->n_tiles_bwd, kStreamThreads, s, sys, b->tile_bwd.as<uint64_t>(), b->n);
    }
  }
  count_launch();
  batch_scatter_kernel<<<rows, 256, 0, s>>>(sys);
  MCS_LAUNCHED();
  return MC_OK;
}

int batch_mlem(mc_batch *b, int n_iter, cudaStream_t s) {
  if (!b->exec || b->exec_iters != n_iter) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    cudaStream_t cap = nullptr;
    MCS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = MC_OK;
    if (e == cudaSuccess) {
      rc = batch_enqueue(b, n_iter, cap);
      e = cudaStreamEndCapture(cap, &g);
    }
    if (e == cudaSuccess && rc == MC_OK) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (rc != MC_OK) return rc;
    if (e != cudaSuccess) { set_error("batch graph capture failed: %s", cudaGetErrorString(e)); return MC_ECUDA; }
    b->exec_iters = n_iter;
  }
  MCS_CUDA(cudaGraphLaunch(b->exec, s));
  return MC_OK;
}

// The batched reconstruction with the iterations in one cooperative launch
// (start images, iterations, write-back: five launches in all).
int batch_mlem_persistent(mc_batch *b, int n_iter, cudaStream_t s) {
  int dev = 0, coop = 0, per_sm = 0;
  MCS_CUDA(cudaGetDevice(&dev));
  MCS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) { set_error("the device does not support cooperative launches"); return MC_ECUDA; }
  MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel, kStreamThreads, 0));
  if (per_sm < 1) { set_error("the persistent batch kernel does not fit on an SM"); return MC_ECUDA; }
  const BatchSys *sys = b->systems.as<BatchSys>();
  const unsigned rows = (unsigned)(b->n * kInitChunks);
  count_launch();
  batch_init_sums_kernel<<<rows, 256, 0, s>>>(sys, b->part_y.as<double>());
  count_launch();
  batch_init_total_kernel<<<div_up(b->n, 256), 256, 0, s>>>(b->part_y.as<double>(), b->part_s.as<double>(), b->n,
                                                            b->x0.as<double>());
  count_launch();
  batch_init_fill_kernel<<<rows, 256, 0, s>>>(sys, b->x0.as<double>());
  MCS_LAUNCHED();
  if (n_iter > 0 && (b->n_tiles_fwd || b->n_tiles_bwd)) {
    // every block resident (a grid-wide barrier needs all of them); no more
    // blocks than tiles of the larger half
    uint64_t grid = (uint64_t)per_sm * (uint64_t)device_sm_count();
    const uint64_t most = std::max(b->n_tiles_fwd, b->n_tiles_bwd);
    if (grid > most) grid = most;
    const uint64_t *tf = b->tile_fwd.as<uint64_t>(), *tb = b->tile_bwd.as<uint64_t>();
    uint64_t nf = b->n_tiles_fwd, nb = b->n_tiles_bwd;
    int n_sys = b->n, it = n_iter;
    void *args[] = {(void *)&sys, (void *)&tf, (void *)&nf, (void *)&tb, (void *)&nb, (void *)&n_sys, (void *)&it};
    count_launch();
    MCS_CUDA(cudaLaunchCooperativeKernel((const void *)batch_persistent_kernel, dim3((unsigned)grid),
                                         dim3(kStreamThreads), args, 0, s));
  }
  count_launch();
  batch_scatter_kernel<<<rows, 256, 0, s>>>(sys);
  MCS_LAUNCHED();
  return MC_OK;
}

void batch_free(mc_batch *b) { delete b; }

// ---------------------------------------------------------------------------
// SpMV autotuner: per system, the fastest of the streaming tiles and the row
// groups of 1..32 lanes, for the forward and the back-projection separately
// ---------------------------------------------------------------------------
int autotune(mc_system *sys, cudaStream_t s, int *fwd_choice, int *bwd_choice) {
  if (sys->n_rows == 0 || sys->n_cols == 0 || sys->nnz == 0) { *fwd_choice = *bwd_choice = -1; return MC_OK; }
  cudaEvent_t a = nullptr, b = nullptr;
  MCS_CUDA(cudaEventCreate(&a));
  MCS_CUDA(cudaEventCreate(&b));
  const int64_t fwd_tiles = sys->n_csr_blocks, bwd_tiles = sys->n_csc_blocks;
  const int g_fwd0 = sys->spmv_group_fwd, g_bwd0 = sys->spmv_group_bwd;
  float best_f = 1e30f, best_b = 1e30f;
  int choice_f = -1, choice_b = -1;
  const int groups[6] = {1, 2, 4, 8, 16, 32};
  for (int c = -1; c < 6; ++c) {  // -1: streaming tiles
    if (c == -1 && fwd_tiles == 0 && bwd_tiles == 0) continue;
    sys->n_csr_blocks = c == -1 ? fwd_tiles : 0;
    sys->n_csc_blocks = c == -1 ? bwd_tiles : 0;
    if (c >= 0) { sys->spmv_group_fwd = groups[c]; sys->spmv_group_bwd = groups[c]; }
    for (int pass = 0; pass < 2; ++pass) {  // warm-up, then timed
      float tf = 0.f, tb = 0.f;
      if (c >= 0 || fwd_tiles) {
        cudaEventRecord(a, s);
        for (int r = 0; r < 5; ++r) fwd_dispatch<0, false>(sys, sys->xs.as<float>(), nullptr, sys->r.as<float>(), nullptr, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&tf, a, b);
        if (pass && tf < best_f) { best_f = tf; choice_f = c; }
      }
      if (c >= 0 || bwd_tiles) {
        cudaEventRecord(a, s);
        for (int r = 0; r < 5; ++r) back_dispatch<0>(sys, sys->r.as<float>(), sys->xs.as<float>(), nullptr, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&tb, a, b);
        if (pass && tb < best_b) { best_b = tb; choice_b = c; }
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  MCS_LAUNCHED();
  sys->n_csr_blocks = choice_f == -1 ? fwd_tiles : 0;
  sys->n_csc_blocks = choice_b == -1 ? bwd_tiles : 0;
  sys->spmv_group_fwd = choice_f >= 0 ? groups[choice_f] : g_fwd0;
  sys->spmv_group_bwd = choice_b >= 0 ? groups[choice_b] : g_bwd0;
  // partials must cover the forward blocks of the chosen kernel
  const int fb = forward_blocks(sys);
  if ((size_t)fb * sizeof(double) > sys->partials.bytes) MCS_TRY(sys->partials.alloc((size_t)fb * sizeof(double), s));
  *fwd_choice = choice_f == -1 ? 0 : groups[choice_f];
  *bwd_choice = choice_b == -1 ? 0 : groups[choice_b];
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

}  // namespace mcs
