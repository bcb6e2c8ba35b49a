// internal.cuh -- declarations shared by the translation units of
// libmcspect.so (not part of the public ABI; see include/mcspect.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/mcspect.h"

namespace mcs {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();
// Counts kernel launches made by this library (reported by mc_kernel_launches).
void count_launch();

#define MCS_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      ::mcs::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA;                          \
    }                                                                                         \
  } while (0)

#define MCS_LAUNCHED()                                                                        \
  do {                                                                                        \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess) {                                                                  \
      ::mcs::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return MC_ECUDA;                                                                        \
    }                                                                                         \
  } while (0)

#define MCS_TRY(expr)            \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != MC_OK) return rc_; \
  } while (0)

// Device buffer owned by host code; freed on destruction (stream-ordered).
// Once per device: let the stream-ordered allocator's default pool keep up
// to 32 GiB of freed memory (instead of returning it to the driver
// at every synchronisation), so that the large, short-lived buffers of a
// build are not mapped afresh each time.  Process-local; ends with it.
void keep_pool_memory();

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; o.bytes = 0; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; s = o.s; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  int alloc(size_t n, cudaStream_t stream) {
    release();
    s = stream;
    bytes = n;
    if (n == 0) return MC_OK;
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(&p, n, stream);
    if (e != cudaSuccess) {
      p = nullptr;
      bytes = 0;
      set_error("device allocation of %zu bytes failed: %s", n, cudaGetErrorString(e));
      return MC_ENOMEM;
    }
    return MC_OK;
  }
  void release() {
    if (p && cudaFreeAsync(p, s) != cudaSuccess) {
      (void)cudaGetLastError();  // e.g. the allocating stream is gone
      cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// the system matrix (device resident)
// ---------------------------------------------------------------------------
}  // namespace mcs

struct mc_system {
  // the device current when the system was made: its buffers live there
  mc_system() {
    if (cudaGetDevice(&device) != cudaSuccess) device = -1;
  }
  int device = -1;
  int64_t n_rows = 0, n_cols = 0, nnz = 0, n_events = 0;
  uint64_t first = 0, count = 0;
  uint64_t fates[4] = {0, 0, 0, 0};
  uint32_t max_count = 0;
  int32_t value_type = MC_VAL_F32;
  double ms_transport = 0.0, ms_detect = 0.0, ms_assembly = 0.0;
  // CSR (rows -> cols) and CSC (cols -> rows) of the counts C_jv
  mcs::DevBuf row_ptr, col_idx, csr_cnt;  // u32 [M+1], u32 [nnz], u32 [nnz]
  mcs::DevBuf col_ptr, row_idx, csc_cnt;  // u32 [N+1], u32 [nnz], u32 [nnz]
  // projector values (counts as float / half / bfloat16)
  mcs::DevBuf csr_val, csc_val;
  mcs::DevBuf n_v;      // u32 [N]: histories started in voxel v
  mcs::DevBuf inv_n;    // f32 [N]: 1/n_v (0 if n_v = 0)
  mcs::DevBuf colsum;   // f64 [N]: S_v = sum_j C_jv
  mcs::DevBuf inv_colsum;  // f32 [N]: 1/S_v (0 if S_v = 0)
  // Stored values that are not the exact counts: for the rounded-A value
  // types (MC_VAL_F16_A, MC_VAL_BF16_A) the values are A itself, so the
  // image is not prescaled (ones) and the normaliser is the stored matrix's
  // column sum s~_v; for counts rounded to half / bfloat16 (allow_rounding)
  // the normaliser is the column sum S~_v of the rounded counts.  Either
  // way ML-EM runs on the matrix the projectors read.
  bool rounded_counts = false;
  mcs::DevBuf a_ones;        // f32 [N]: 1
  mcs::DevBuf a_sens;        // f64 [N]: s~_v = sum_j val_jv (A types) or S~_v (rounded counts)
  mcs::DevBuf a_inv_sens;    // f32 [N]: its reciprocal (0 if 0)
  // work vectors of the projectors / ML-EM
  mcs::DevBuf xs;       // f32 [N]: x_v / n_v
  mcs::DevBuf r;        // f32 [M]
  mcs::DevBuf partials; // f64 [max blocks]
  mcs::DevBuf ll;       // f64 [ll_cap]
  int64_t ll_cap = 0;
  int spmv_group_fwd = 4, spmv_group_bwd = 4;  // lanes per row / per column
  // tile partition of the non-zeros for the streaming SpMV kernels (empty:
  // fall back to the row-group kernels)
  mcs::DevBuf csr_blocks, csc_blocks;  // u32 [n_blocks + 1] first row / column of each tile
  int64_t n_csr_blocks = 0, n_csc_blocks = 0;
  bool warp_rows_fwd = false, warp_rows_bwd = false;
  // forced detection: the entries are summed event weights instead of
  // counts, in fixed point (q * 2^-48); the counts above are then the
  // number of weighted events per entry
  bool weighted = false;
  mcs::DevBuf csr_wq, csc_wq;  // u64 [nnz]
  // ordered subsets: row i of this system is row row_map[i] of its parent
  // (empty for a full system)
  mcs::DevBuf row_map;
  int64_t parent_rows = 0;
  int32_t n_subsets = 1, subset = 0;
};

struct mc_batch;

namespace mcs {

// value types: storage (0 float, 1 half, 2 bfloat16) and whether the stored
// values are A = C diag(1/n_v) itself rather than the counts C
inline int value_storage(int vt) { return vt == MC_VAL_F16 || vt == MC_VAL_F16_A ? 1 : vt == MC_VAL_F32 ? 0 : 2; }
inline bool values_are_a(int vt) { return vt == MC_VAL_F16_A || vt == MC_VAL_BF16_A; }
// Scale applied to the image before the forward projection (1/n_v for
// count values, 1 for A values), the back-projection's normaliser (1/S_v,
// or 1/s~_v) and the sensitivity terms the start image sums (S_v with
// per-voxel division by n_v, or s~_v as it is: n_v pointer NULL).
inline const float *proj_scale(const mc_system *s) {
  return values_are_a(s->value_type) ? s->a_ones.as<float>() : s->inv_n.as<float>();
}
inline const float *proj_inv_norm(const mc_system *s) {
  return values_are_a(s->value_type) || s->rounded_counts ? s->a_inv_sens.as<float>() : s->inv_colsum.as<float>();
}
inline const double *proj_sens_terms(const mc_system *s, const uint32_t **n_v) {
  if (values_are_a(s->value_type)) { *n_v = nullptr; return s->a_sens.as<double>(); }
  *n_v = s->n_v.as<uint32_t>();
  return s->rounded_counts ? s->a_sens.as<double>() : s->colsum.as<double>();
}

// ---------------------------------------------------------------------------
// build pieces implemented in the .cu files
// ---------------------------------------------------------------------------

// Host-side description of one transport launch (built in api.cu).
struct TransportSetup {
  // grid
  int nx, ny, nz;
  double h;
  const uint8_t *material_dev;
  int n_mat;
  double rho[256], zoa[256], zeff[256];
  // camera
  int n_views, bins_u, bins_v;
  double start_deg, arc_deg, bin_mm, radius_mm, hole_len, hole_diam, fwhm, e0, window, photo_k;
  const double *view_cs_dev;  // [2*V]: cos, sin of theta_k (double)
  const float *view_cs_f_dev; // [2*V] same, float
  const double *coef_d_dev;   // [3*n_mat] 0.1 rho, N_A Z/A, k Z^4 (double)
  const float *coef_f_dev;    // [3*n_mat] 0.1 rho N_A Z/A, 0.1 rho k Z^4, 0 (float)
  const float *sig_tab_dev;   // float path: sigma_KN over the energy window
  const uint8_t *skip_dev;    // float forced detection: distance map (see build_skip_map), else null
  // run
  uint64_t first, count;
  uint32_t key0, key1;
  // outputs
  unsigned long long *events;  // key = v*M + j
  unsigned long long capacity;
  unsigned long long *cursor;
  unsigned long long *fates;   // [4]
  mc_history_record *records;  // trace mode (else null)
  void *esc;                   // escape queue (EscapeRec of the precision)
  unsigned long long esc_capacity;
  unsigned long long *esc_cursor;
  cudaEvent_t ev_mid;          // recorded between transport and detection (optional)
  int precision;
  int primary_only;            // tally only unscattered photons
  int forced;                  // forced detection: weighted copies instead of analog detection
  int forced_dir;              // forced emission direction (primary tally): weighted analog detections
  unsigned long long *weights; // forced detection: fixed-point weight of each event (else null)
};

// Distance map of a material grid for the float forced-detection traversal:
// skip[v] = the largest D <= kSkipCap such that every voxel of the grid within
// chessboard distance D - 1 of v holds v's material (voxels outside the grid
// do not count).  A ray inside voxel v stays in that cube of constant mu until
// it crosses one of the cube's faces, so the traversal can cross it in one step.
constexpr int kSkipCap = 16;
int build_skip_map(const uint8_t *material, int nx, int ny, int nz, uint8_t *skip, cudaStream_t s);

// forced detection: event weights are tallied as q = rint(w * 2^48)
constexpr double kFdScale = 281474976710656.0;

// bytes of one forced-detection interaction record for a precision
inline size_t fd_rec_bytes(int precision) { return precision == MC_FP64 ? 80 : 48; }

// bytes of one escape-queue entry for a precision
inline size_t escape_rec_bytes(int precision) { return precision == MC_FP64 ? 64 : 40; }

int launch_transport(const TransportSetup &ts, cudaStream_t s);
int launch_debug_kn(double e_kev, int precision, uint64_t seed, uint64_t n, double *cos_dev, double *eps_dev,
                    cudaStream_t s);
int launch_debug_beam(const TransportSetup &ts, uint64_t n, const double p0[3], const double d[3], double e_kev,
                      unsigned long long *through_dev, cudaStream_t s);

// Assembly: sorted events -> CSR + CSC + n_v + column sums.  `keys` holds
// n keys (v*M + j) and is overwritten.
// `weights` (device, optional): fixed-point weight of each event; the
// entries are then the weight sums (the system is marked weighted).
int assemble_system(mc_system *sys, DevBuf &keys, int64_t n, cudaStream_t s, const uint64_t *weights = nullptr);

// Projector value arrays for sys->value_type.
int make_values(mc_system *sys, cudaStream_t s);
int set_spmv_layout(mc_system *sys, int fwd, int bwd, cudaStream_t s);

// System of the rows of views subset, subset + n_sub, ... of a parent whose
// rows are view-major with rpv rows per view (assemble.cu).
int subset_system(const mc_system *parent, int64_t rpv, int n_sub, int subset, mc_system *sys, cudaStream_t s);

// Tile partition of CSR and CSC for the streaming SpMV kernels (mlem.cu).
int make_stream_blocks(mc_system *sys, cudaStream_t s);

// Scans / sorts (assemble.cu)
int exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, cudaStream_t s);
// Stable LSD radix sort of keys (and payload) on bits [first_bit, bits) of
// the keys; the result is in keys/vals or, if *result_in_alt, in the alts.
int radix_sort_u64(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n, int bits,
                   bool *result_in_alt, cudaStream_t s, int first_bit = 0);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of
//   (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0))
// with the key bumped by the Weyl increments after each round.
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// One history's stream: block b of history h is counter (b, 0, h_lo, h_hi)
// under key (seed_lo, seed_hi); words are consumed w0, w1, w2, w3, then the
// next block.
struct Stream {
  uint32_t k0, k1, h_lo, h_hi;
  uint32_t block;
  uint32_t w0, w1, w2, w3;
  uint32_t left;
  uint32_t n_draws;
  __device__ __forceinline__ void init(uint32_t key0, uint32_t key1, uint64_t h) {
    k0 = key0; k1 = key1;
    h_lo = (uint32_t)h; h_hi = (uint32_t)(h >> 32);
    block = 0; left = 0; n_draws = 0;
  }
  __device__ __forceinline__ uint32_t word() {
    if (left == 0) {
      uint32_t c0 = block, c1 = 0u, c2 = h_lo, c3 = h_hi;
      philox4x32_10(c0, c1, c2, c3, k0, k1);
      w0 = c0; w1 = c1; w2 = c2; w3 = c3;
      block += 1;
      left = 4;
    }
    const uint32_t w = w0;
    w0 = w1; w1 = w2; w2 = w3;
    left -= 1;
    n_draws += 1;
    return w;
  }
};

// Uniform in (0,1).  double: (w + 1/2) 2^-32 (exact).  float: the top 23
// bits, (floor(w / 2^9) + 1/2) 2^-23, computed as ((w >> 8) | 1) 2^-24
// (an odd 24-bit integer, exact in float).
template <typename T> __device__ __forceinline__ T uniform(uint32_t w);
template <> __device__ __forceinline__ double uniform<double>(uint32_t w) {
  return ((double)w + 0.5) * (1.0 / 4294967296.0);
}
// ((w >> 8) | 1) 2^-24 = ((w >> 9) + 1/2) 2^-23, built from the bits: the
// float 1 + (w >> 9) 2^-23, minus 1, plus 2^-24 (every step exact)
template <> __device__ __forceinline__ float uniform<float>(uint32_t w) {
  return (__uint_as_float(0x3F800000u | (w >> 9)) - 1.0f) + 5.9604644775390625e-8f;
}

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

int device_sm_count();

}  // namespace mcs
