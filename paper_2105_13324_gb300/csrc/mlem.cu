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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

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

// MODE 0: out = q.  MODE 1: out = r = y / q (0 where q = 0), and with LL the
// block's share of sum_j (y_j ln q_j - q_j) in partials[blockIdx.x].
template <typename V, int G, int MODE, bool LL>
__global__ void __launch_bounds__(kSpmvThreads) csr_forward_kernel(const uint32_t *__restrict__ row_ptr,
                                                                   const uint32_t *__restrict__ col,
                                                                   const V *__restrict__ val,
                                                                   const float *__restrict__ xs, int64_t m,
                                                                   const float *__restrict__ y,
                                                                   float *__restrict__ out, double *partials) {
  __shared__ double s_tmp[kSpmvThreads / 32];
  const int64_t gid = ((int64_t)blockIdx.x * kSpmvThreads + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  double ll = 0.0;
  // every lane takes part in the shuffles; lanes past the last row see an
  // empty range
  uint32_t b = 0, e = 0;
  if (gid < m) { b = row_ptr[gid]; e = row_ptr[gid + 1]; }
  float acc = 0.0f;
  for (uint32_t k = b + sub; k < e; k += G) acc = fmaf(to_f(val[k]), __ldg(xs + col[k]), acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
  if (gid < m && sub == 0) {
    if (MODE == 0) {
      out[gid] = acc;
    } else {
      const float yj = y[gid];
      out[gid] = acc > 0.0f ? yj / acc : 0.0f;
      if (LL) ll = (yj > 0.0f ? (double)yj * log((double)acc) : 0.0) - (double)acc;
    }
  }
  if (LL) {
    const double t = block_sum_double(ll, s_tmp);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// MODE 0: out_v = (1/n_v) sum_j C_jv r_j (back-projection A^T r).
// MODE 1: x_v <- x_v t_v / S_v (0 where S_v = 0), xs_v = x_v / n_v.
template <typename V, int G, int MODE>
__global__ void __launch_bounds__(kSpmvThreads) csc_back_kernel(const uint32_t *__restrict__ col_ptr,
                                                                const uint32_t *__restrict__ row,
                                                                const V *__restrict__ val,
                                                                const float *__restrict__ r, int64_t n,
                                                                const float *__restrict__ inv_n,
                                                                const float *__restrict__ inv_colsum,
                                                                float *__restrict__ x, float *__restrict__ xs) {
  const int64_t gid = ((int64_t)blockIdx.x * kSpmvThreads + threadIdx.x) / G;
  const int sub = threadIdx.x & (G - 1);
  uint32_t b = 0, e = 0;
  if (gid < n) { b = col_ptr[gid]; e = col_ptr[gid + 1]; }
  float acc = 0.0f;
  for (uint32_t k = b + sub; k < e; k += G) acc = fmaf(to_f(val[k]), __ldg(r + row[k]), acc);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
  if (gid < n && sub == 0) {
    if (MODE == 0) {
      x[gid] = acc * inv_n[gid];
    } else {
      const float is = inv_colsum[gid];
      const float xn = is > 0.0f ? x[gid] * acc * is : 0.0f;
      x[gid] = xn;
      xs[gid] = xn * inv_n[gid];
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

// partials[b] = block b's sum of y (double) and of s_v = S_v / n_v
__global__ void init_sums_kernel(const float *y, int64_t m, const double *colsum, const uint32_t *n_v, int64_t n,
                                 double *py, double *ps) {
  __shared__ double s_tmp[32];
  double ay = 0.0, as = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    ay += (double)y[i];
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (n_v[v]) as += colsum[v] / (double)n_v[v];
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
    s[v] = n_v[v] ? colsum[v] / (double)n_v[v] : 0.0;
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
static int grid_stride_blocks(int64_t n) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = (int64_t)device_sm_count() * 16;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <typename V, int MODE, bool LL>
static void fwd_launch(const mc_system *sys, int g, const float *xs, const float *y, float *out, double *partials,
                       cudaStream_t s) {
  const int64_t m = sys->n_rows;
  const int blocks = div_up(m * g, kSpmvThreads);
  const V *val = sys->csr_val.as<V>();
  const uint32_t *rp = sys->row_ptr.as<uint32_t>(), *ci = sys->col_idx.as<uint32_t>();
  switch (g) {
    case 1: count_launch(); csr_forward_kernel<V, 1, MODE, LL><<<blocks, kSpmvThreads, 0, s>>>(rp, ci, val, xs, m, y, out, partials); break;
    case 2: count_launch(); csr_forward_kernel<V, 2, MODE, LL><<<blocks, kSpmvThreads, 0, s>>>(rp, ci, val, xs, m, y, out, partials); break;
    case 4: count_launch(); csr_forward_kernel<V, 4, MODE, LL><<<blocks, kSpmvThreads, 0, s>>>(rp, ci, val, xs, m, y, out, partials); break;
    case 8: count_launch(); csr_forward_kernel<V, 8, MODE, LL><<<blocks, kSpmvThreads, 0, s>>>(rp, ci, val, xs, m, y, out, partials); break;
    case 16: count_launch(); csr_forward_kernel<V, 16, MODE, LL><<<blocks, kSpmvThreads, 0, s>>>(rp, ci, val, xs, m, y, out, partials); break;
    default: count_launch(); csr_forward_kernel<V, 32, MODE, LL><<<blocks, kSpmvThreads, 0, s>>>(rp, ci, val, xs, m, y, out, partials); break;
  }
}

template <typename V, int MODE>
static void back_launch(const mc_system *sys, int g, const float *r, float *x, float *xs, cudaStream_t s) {
  const int64_t n = sys->n_cols;
  const int blocks = div_up(n * g, kSpmvThreads);
  const V *val = sys->csc_val.as<V>();
  const uint32_t *cp = sys->col_ptr.as<uint32_t>(), *ri = sys->row_idx.as<uint32_t>();
  const float *inv_n = sys->inv_n.as<float>(), *ics = sys->inv_colsum.as<float>();
  switch (g) {
    case 1: count_launch(); csc_back_kernel<V, 1, MODE><<<blocks, kSpmvThreads, 0, s>>>(cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 2: count_launch(); csc_back_kernel<V, 2, MODE><<<blocks, kSpmvThreads, 0, s>>>(cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 4: count_launch(); csc_back_kernel<V, 4, MODE><<<blocks, kSpmvThreads, 0, s>>>(cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 8: count_launch(); csc_back_kernel<V, 8, MODE><<<blocks, kSpmvThreads, 0, s>>>(cp, ri, val, r, n, inv_n, ics, x, xs); break;
    case 16: count_launch(); csc_back_kernel<V, 16, MODE><<<blocks, kSpmvThreads, 0, s>>>(cp, ri, val, r, n, inv_n, ics, x, xs); break;
    default: count_launch(); csc_back_kernel<V, 32, MODE><<<blocks, kSpmvThreads, 0, s>>>(cp, ri, val, r, n, inv_n, ics, x, xs); break;
  }
}

template <int MODE, bool LL>
static void fwd_dispatch(const mc_system *sys, const float *xs, const float *y, float *out, double *partials,
                         cudaStream_t s) {
  const int g = sys->spmv_group_fwd;
  if (sys->value_type == MC_VAL_F16) fwd_launch<__half, MODE, LL>(sys, g, xs, y, out, partials, s);
  else if (sys->value_type == MC_VAL_BF16) fwd_launch<__nv_bfloat16, MODE, LL>(sys, g, xs, y, out, partials, s);
  else fwd_launch<float, MODE, LL>(sys, g, xs, y, out, partials, s);
}

template <int MODE>
static void back_dispatch(const mc_system *sys, const float *r, float *x, float *xs, cudaStream_t s) {
  const int g = sys->spmv_group_bwd;
  if (sys->value_type == MC_VAL_F16) back_launch<__half, MODE>(sys, g, r, x, xs, s);
  else if (sys->value_type == MC_VAL_BF16) back_launch<__nv_bfloat16, MODE>(sys, g, r, x, xs, s);
  else back_launch<float, MODE>(sys, g, r, x, xs, s);
}

int forward_blocks(const mc_system *sys) { return div_up(sys->n_rows * sys->spmv_group_fwd, kSpmvThreads); }

int project(const mc_system *sys, const float *x, float *q, cudaStream_t s) {
  if (sys->n_cols > 0) {
    count_launch(); prescale_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(x, sys->inv_n.as<float>(), sys->xs.as<float>(),
                                                                     sys->n_cols);
  }
  if (sys->n_rows > 0) fwd_dispatch<0, false>(sys, sys->xs.as<float>(), nullptr, q, nullptr, s);
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
    count_launch(); sensitivity_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(sys->colsum.as<double>(),
                                                                       sys->n_v.as<uint32_t>(), sys->n_cols, out);
  }
  MCS_LAUNCHED();
  return MC_OK;
}

int mlem_init(mc_system *sys, const float *y, float *x, cudaStream_t s) {
  const int nb = 256;
  DevBuf part;
  MCS_TRY(part.alloc((2 * nb + 1) * sizeof(double), s));
  double *py = part.as<double>(), *ps = py + nb, *x0 = py + 2 * nb;
  count_launch();
  init_sums_kernel<<<nb, 256, 0, s>>>(y, sys->n_rows, sys->colsum.as<double>(), sys->n_v.as<uint32_t>(), sys->n_cols,
                                      py, ps);
  count_launch();
  init_total_kernel<<<1, 256, 0, s>>>(py, ps, nb, x0);
  MCS_LAUNCHED();
  if (sys->n_cols > 0) {
    count_launch();
    init_fill_kernel<<<grid_stride_blocks(sys->n_cols), 256, 0, s>>>(x0, sys->colsum.as<double>(),
                                                                     sys->inv_n.as<float>(), sys->n_cols, x,
                                                                     sys->xs.as<float>());
  }
  MCS_LAUNCHED();
  return MC_OK;
}

int mlem_run(mc_system *sys, const float *y, float *x, int n_iter, bool want_ll, cudaStream_t s) {
  const int64_t m = sys->n_rows, n = sys->n_cols;
  if (n > 0) {
    count_launch(); prescale_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x, sys->inv_n.as<float>(), sys->xs.as<float>(), n);
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
    prescale_kernel<<<grid_stride_blocks(n), 256, 0, s>>>(x_dev, sys->inv_n.as<float>(), xs, n);
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
