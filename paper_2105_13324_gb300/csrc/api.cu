// api.cu -- the extern "C" entry points of libmcspect.so (include/mcspect.h):
// argument checks, the build pipeline (transport -> assembly -> values) and
// the projector / ML-EM calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace mcs {

static thread_local std::string g_error;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
}

void clear_error() { g_error.clear(); }

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int device_sm_count() {
  static std::mutex mu;
  static std::vector<int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cache[dev] = n;
  }
  return cache[dev];
}

void keep_pool_memory() {
  static std::mutex mu;
  static std::vector<char> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)done.size() <= dev) done.resize(dev + 1, 0);
  if (done[dev]) return;
  done[dev] = 1;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) { (void)cudaGetLastError(); return; }
  uint64_t keep = 32ull << 30;  // 32 GiB
  if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) (void)cudaGetLastError();
}

int launch_transport_f32(const TransportSetup &ts, cudaStream_t s);
int launch_transport_f64(const TransportSetup &ts, cudaStream_t s);
int launch_debug_kn_f32(double e, uint64_t seed, uint64_t n, double *c, double *p, cudaStream_t s);
int launch_debug_kn_f64(double e, uint64_t seed, uint64_t n, double *c, double *p, cudaStream_t s);
int launch_debug_beam_f32(const TransportSetup &ts, uint64_t n, const double p0[3], const double d[3], double e,
                          unsigned long long *t, cudaStream_t s);
int launch_debug_beam_f64(const TransportSetup &ts, uint64_t n, const double p0[3], const double d[3], double e,
                          unsigned long long *t, cudaStream_t s);

int project(const mc_system *sys, const float *x, float *q, cudaStream_t s);
int backproject(const mc_system *sys, const float *r, float *b, cudaStream_t s);
int sensitivity(const mc_system *sys, double *out, cudaStream_t s);
int mlem_init(mc_system *sys, const float *y, float *x, cudaStream_t s);
int mlem_run(mc_system *sys, const float *y, float *x, int n_iter, bool want_ll, cudaStream_t s);
int osem_run(mc_system *const *fwd, mc_system *const *back, int n_sub, const float *y, const float *add, float *x,
             int n_iter, cudaStream_t s);
int forward_blocks(const mc_system *sys);
int project_f64(const mc_system *sys, const double *x, double *q, cudaStream_t s);
int project_ratio(const mc_system *sys, const float *x, const float *y, float *r, cudaStream_t s);
int loglik(const mc_system *sys, const float *x, const float *y, double *value, cudaStream_t s);
int backproject_f64(const mc_system *sys, const double *r, double *b, cudaStream_t s);
template <typename T>
int prior_quadratic(int nx, int ny, int nz, double beta, const T *x, T *grad, double *value, cudaStream_t s);
int pgd_step(int64_t n, double alpha, const double *sens, const float *bp, const float *gp, float *x, cudaStream_t s);
int batch_create(mc_system *const *sys, int n, const float *const *y, float *const *x, mc_batch **out);
int batch_mlem(mc_batch *b, int n_iter, cudaStream_t s);
int batch_mlem_persistent(mc_batch *b, int n_iter, cudaStream_t s);
void batch_free(mc_batch *b);
int autotune(mc_system *sys, cudaStream_t s, int *fwd_choice, int *bwd_choice);
int vector_sum(int64_t n, const float *v, double *out, cudaStream_t s);
int mlem_start(int64_t n, const double *sens, double sum_y, float *x, cudaStream_t s);
void compute_coefficients(const TransportSetup &ts, std::vector<double> &cd, std::vector<float> &cf,
                          std::vector<float> &sig_tab);

static constexpr double kPiHost = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static int check_phantom(const mc_phantom *ph) {
  if (!ph) { set_error("phantom is NULL"); return MC_EINVAL; }
  if (ph->nx < 1 || ph->ny < 1 || ph->nz < 1) { set_error("grid dimensions must be positive"); return MC_EINVAL; }
  const uint64_t nv = (uint64_t)ph->nx * ph->ny * ph->nz;
  if (nv >= (1ull << 31)) { set_error("grid of %llu voxels exceeds 2^31", (unsigned long long)nv); return MC_EINVAL; }
  if (!(ph->voxel_mm > 0.0) || !std::isfinite(ph->voxel_mm)) { set_error("voxel_mm must be positive"); return MC_EINVAL; }
  if (!ph->material_host || !ph->rho_host || !ph->z_over_a_host || !ph->z_eff_host) {
    set_error("phantom arrays must not be NULL");
    return MC_EINVAL;
  }
  if (ph->n_materials < 1 || ph->n_materials > 256) { set_error("n_materials must be in 1..256"); return MC_EINVAL; }
  for (int m = 0; m < ph->n_materials; ++m) {
    if (!(ph->rho_host[m] >= 0.0) || !(ph->z_over_a_host[m] >= 0.0) || !(ph->z_eff_host[m] >= 0.0) ||
        !std::isfinite(ph->rho_host[m]) || !std::isfinite(ph->z_over_a_host[m]) || !std::isfinite(ph->z_eff_host[m])) {
      set_error("material %d has a negative or non-finite property", m);
      return MC_EINVAL;
    }
  }
  for (uint64_t i = 0; i < nv; ++i) {
    if (ph->material_host[i] >= ph->n_materials) {
      set_error("voxel %llu has material %d outside the table", (unsigned long long)i, (int)ph->material_host[i]);
      return MC_EINVAL;
    }
  }
  return MC_OK;
}

static int check_geometry(const mc_geometry *g, const mc_phantom *ph) {
  if (!g) { set_error("geometry is NULL"); return MC_EINVAL; }
  if (g->n_views < 1 || g->n_bins_u < 1 || g->n_bins_v < 1) { set_error("views and bins must be positive"); return MC_EINVAL; }
  const uint64_t m = (uint64_t)g->n_views * g->n_bins_u * g->n_bins_v;
  if (m >= (1ull << 31)) { set_error("%llu detector rows exceed 2^31", (unsigned long long)m); return MC_EINVAL; }
  const double vals[] = {g->start_deg, g->arc_deg, g->bin_mm, g->radius_mm, g->hole_len_mm, g->hole_diam_mm,
                         g->fwhm_mm, g->e0_kev, g->window_frac, g->photo_k};
  for (double v : vals)
    if (!std::isfinite(v)) { set_error("geometry has a non-finite value"); return MC_EINVAL; }
  if (!(g->bin_mm > 0) || !(g->hole_len_mm > 0) || !(g->hole_diam_mm > 0) || !(g->fwhm_mm >= 0) || !(g->e0_kev > 0) ||
      !(g->window_frac > 0 && g->window_frac < 2) || !(g->photo_k >= 0) || !(g->arc_deg > 0)) {
    set_error("geometry values out of range");
    return MC_EINVAL;
  }
  if (g->precision != MC_FP32 && g->precision != MC_FP64) { set_error("precision must be MC_FP32 or MC_FP64"); return MC_EINVAL; }
  if (g->tally < 0 || g->tally > (MC_TALLY_PRIMARY | MC_TALLY_FORCED | MC_TALLY_FORCED_DIRECTION)) {
    set_error("tally must be MC_TALLY_ALL or MC_TALLY_PRIMARY, optionally with MC_TALLY_FORCED or "
              "MC_TALLY_FORCED_DIRECTION");
    return MC_EINVAL;
  }
  if ((g->tally & MC_TALLY_FORCED_DIRECTION) &&
      (!(g->tally & MC_TALLY_PRIMARY) || (g->tally & MC_TALLY_FORCED))) {
    set_error("MC_TALLY_FORCED_DIRECTION goes with MC_TALLY_PRIMARY only (it is exact for unscattered photons; "
              "forced detection's emission copies do not depend on the direction)");
    return MC_EINVAL;
  }
  if (ph) {
    const double hx = 0.5 * ph->nx * ph->voxel_mm, hy = 0.5 * ph->ny * ph->voxel_mm;
    if (!(g->radius_mm > std::sqrt(hx * hx + hy * hy))) {
      set_error("collimator front face (radius %.3f mm) must clear the grid (half-diagonal %.3f mm)", g->radius_mm,
                std::sqrt(hx * hx + hy * hy));
      return MC_EINVAL;
    }
  }
  return MC_OK;
}

}  // namespace mcs

// A phantom + geometry resident on the device: the map, the view table and
// the attenuation coefficients, ready for any number of builds.
struct mc_plan {
  mcs::TransportSetup ts;
  mcs::DevBuf material, views_d, views_f, coef_d, coef_f, sig_tab, skip;
};

namespace mcs {

// One pass of the distance map: D(v) = 1 + min over the 26 neighbours u inside
// the grid of (material u == material v ? D(u) : 0), capped.  Starting from
// D = 1 everywhere, pass k gives min(distance, k + 1).
__global__ void skip_pass_kernel(const uint8_t *mat, int nx, int ny, int nz, const uint8_t *din, uint8_t *dout,
                                 int cap) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(v % nx), iy = (int)((v / nx) % ny), iz = (int)(v / ((int64_t)nx * ny));
    const uint8_t m = mat[v];
    int lo = cap - 1;
    for (int dz = -1; dz <= 1; ++dz) {
      const int z = iz + dz;
      if (z < 0 || z >= nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int y = iy + dy;
        if (y < 0 || y >= ny) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int x = ix + dx;
          if (x < 0 || x >= nx || (dx == 0 && dy == 0 && dz == 0)) continue;
          const int64_t u = ((int64_t)z * ny + y) * nx + x;
          const int du = mat[u] == m ? (int)din[u] : 0;
          lo = du < lo ? du : lo;
        }
      }
    }
    dout[v] = (uint8_t)(lo + 1);
  }
}

int build_skip_map(const uint8_t *material, int nx, int ny, int nz, uint8_t *skip, cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny * nz;
  DevBuf tmp;
  MCS_TRY(tmp.alloc((size_t)n, s));
  MCS_CUDA(cudaMemsetAsync(skip, 1, (size_t)n, s));
  int64_t g = (n + 255) / 256;
  if (g > (int64_t)device_sm_count() * 32) g = (int64_t)device_sm_count() * 32;
  uint8_t *a = skip, *b = tmp.as<uint8_t>();
  // kSkipCap - 1 passes (an odd count: the last pass writes into tmp, copied back)
  for (int pass = 0; pass < kSkipCap - 1; ++pass) {
    count_launch();
    skip_pass_kernel<<<(int)g, 256, 0, s>>>(material, nx, ny, nz, a, b, kSkipCap);
    MCS_LAUNCHED();
    uint8_t *t = a; a = b; b = t;
  }
  if (a != skip) MCS_CUDA(cudaMemcpyAsync(skip, a, (size_t)n, cudaMemcpyDeviceToDevice, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

static int prepare_plan(const mc_phantom *ph, const mc_geometry *g, cudaStream_t s, mc_plan &pl) {
  TransportSetup &ts = pl.ts;
  std::memset(&ts, 0, sizeof(ts));
  ts.nx = ph->nx; ts.ny = ph->ny; ts.nz = ph->nz;
  ts.h = ph->voxel_mm;
  ts.n_mat = ph->n_materials;
  for (int m = 0; m < ph->n_materials; ++m) {
    ts.rho[m] = ph->rho_host[m];
    ts.zoa[m] = ph->z_over_a_host[m];
    ts.zeff[m] = ph->z_eff_host[m];
  }
  ts.n_views = g->n_views; ts.bins_u = g->n_bins_u; ts.bins_v = g->n_bins_v;
  ts.start_deg = g->start_deg; ts.arc_deg = g->arc_deg; ts.bin_mm = g->bin_mm; ts.radius_mm = g->radius_mm;
  ts.hole_len = g->hole_len_mm; ts.hole_diam = g->hole_diam_mm; ts.fwhm = g->fwhm_mm;
  ts.e0 = g->e0_kev; ts.window = g->window_frac; ts.photo_k = g->photo_k;
  ts.precision = g->precision;
  ts.primary_only = (g->tally & MC_TALLY_PRIMARY) ? 1 : 0;
  ts.forced = (g->tally & MC_TALLY_FORCED) ? 1 : 0;
  ts.forced_dir = (g->tally & MC_TALLY_FORCED_DIRECTION) ? 1 : 0;
  ts.weights = nullptr;
  const size_t nv = (size_t)ph->nx * ph->ny * ph->nz;
  MCS_TRY(pl.material.alloc(nv, s));
  MCS_CUDA(cudaMemcpyAsync(pl.material.p, ph->material_host, nv, cudaMemcpyHostToDevice, s));
  ts.material_dev = pl.material.as<uint8_t>();
  // view k at theta_k = (start + k (arc / V)) degrees
  std::vector<double> vd(2 * (size_t)g->n_views);
  std::vector<float> vf(2 * (size_t)g->n_views);
  for (int k = 0; k < g->n_views; ++k) {
    const double th = (g->start_deg + k * (g->arc_deg / g->n_views)) * (kPiHost / 180.0);
    vd[2 * k] = std::cos(th);
    vd[2 * k + 1] = std::sin(th);
    vf[2 * k] = (float)vd[2 * k];
    vf[2 * k + 1] = (float)vd[2 * k + 1];
  }
  std::vector<double> cd;
  std::vector<float> cf, tab;
  compute_coefficients(ts, cd, cf, tab);
  MCS_TRY(pl.views_d.alloc(vd.size() * sizeof(double), s));
  MCS_TRY(pl.views_f.alloc(vf.size() * sizeof(float), s));
  MCS_TRY(pl.coef_d.alloc(cd.size() * sizeof(double), s));
  MCS_TRY(pl.coef_f.alloc(cf.size() * sizeof(float), s));
  MCS_TRY(pl.sig_tab.alloc(tab.size() * sizeof(float), s));
  MCS_CUDA(cudaMemcpyAsync(pl.sig_tab.p, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(pl.views_d.p, vd.data(), vd.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(pl.views_f.p, vf.data(), vf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(pl.coef_d.p, cd.data(), cd.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(pl.coef_f.p, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaStreamSynchronize(s));  // host vectors die on return
  ts.view_cs_dev = pl.views_d.as<double>();
  ts.view_cs_f_dev = pl.views_f.as<float>();
  ts.coef_d_dev = pl.coef_d.as<double>();
  ts.coef_f_dev = pl.coef_f.as<float>();
  ts.sig_tab_dev = pl.sig_tab.as<float>();
  ts.skip_dev = nullptr;
  if (ts.forced && ts.precision == MC_FP32) {
    MCS_TRY(pl.skip.alloc(nv, s));
    MCS_TRY(build_skip_map(ts.material_dev, ts.nx, ts.ny, ts.nz, pl.skip.as<uint8_t>(), s));
    ts.skip_dev = pl.skip.as<uint8_t>();
  }
  return MC_OK;
}

static int make_plan(const mc_phantom *ph, const mc_geometry *g, cudaStream_t s, mc_plan **out) {
  MCS_TRY(check_phantom(ph));
  MCS_TRY(check_geometry(g, ph));
  mc_plan *pl = new (std::nothrow) mc_plan();
  if (!pl) { set_error("out of host memory"); return MC_ENOMEM; }
  const int rc = prepare_plan(ph, g, s, *pl);
  if (rc != MC_OK) { delete pl; return rc; }
  *out = pl;
  return MC_OK;
}

static int run_transport(const TransportSetup &ts, cudaStream_t s) {
  return ts.precision == MC_FP64 ? launch_transport_f64(ts, s) : launch_transport_f32(ts, s);
}

// Lanes per row (column) of the row-group kernels from the mean length:
// about 12 or more entries per lane, 16 lanes at most below 1024 entries
// (measured on the 128^3 torso systems: rows of ~70 entries run best with 8
// lanes, rows of ~350 with 16; 32 lanes leave too few loads in flight per
// lane).
static int pick_group(double mean_len) {
  int g = 1;
  while (g < 16 && 12 * g < mean_len) g <<= 1;
  if (mean_len >= 1024.0) g = 32;
  return g;
}

// Work vectors and projector values of a freshly assembled system.
static int finish_system(mc_system *sys, cudaStream_t s) {
  if (sys->parent_rows == 0) sys->parent_rows = sys->n_rows;
  MCS_TRY(make_values(sys, s));
  MCS_TRY(sys->xs.alloc((size_t)(sys->n_cols > 0 ? sys->n_cols : 1) * sizeof(float), s));
  MCS_TRY(sys->r.alloc((size_t)(sys->n_rows > 0 ? sys->n_rows : 1) * sizeof(float), s));
  sys->spmv_group_fwd = pick_group(sys->n_rows > 0 ? (double)sys->nnz / sys->n_rows : 1.0);
  sys->spmv_group_bwd = pick_group(sys->n_cols > 0 ? (double)sys->nnz / sys->n_cols : 1.0);
  MCS_TRY(make_stream_blocks(sys, s));
  const int fb = forward_blocks(sys);
  MCS_TRY(sys->partials.alloc((size_t)(fb > 0 ? fb : 1) * sizeof(double), s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

constexpr int kCounters = 7;  // events, fates[4], queue fill, largest queue fill

__global__ void queue_reset_kernel(unsigned long long *ctr) {
  if (ctr[5] > ctr[6]) ctr[6] = ctr[5];
  ctr[5] = 0ull;
}

// Result of the transport + detection part of a build (the tally, before
// assembly): the event keys v M + j (and, weighted, the fixed-point weights),
// the counters and the device times.
struct Tally {
  DevBuf events, weights;
  unsigned long long hctr[kCounters] = {};
  float ms_transport = 0.f, ms_detect = 0.f;
};

static int tally_from_plan(mc_plan *pl, uint64_t first, uint64_t count, uint64_t seed, cudaStream_t s, Tally &out) {
  if (count == 0) { set_error("no histories requested"); return MC_EINVAL; }
  if (first + count < first) { set_error("history range overflows 64 bits"); return MC_EINVAL; }
  TransportSetup ts = pl->ts;
  ts.first = first;
  ts.count = count;
  ts.key0 = (uint32_t)seed;
  ts.key1 = (uint32_t)(seed >> 32);
  int rc;
  // Histories run in chunks of kChunk: the escape queue is sized for one
  // chunk and reused, the events of all chunks accumulate.  Analog chunks
  // are as long as a queue of at most 4 GiB allows (2^27 .. 2^30
  // histories): every launch of the persistent transport kernel ends in a
  // tail where few warps are left, so fewer, longer launches are faster
  // (10^9 torso histories in one launch instead of eight: 2 % less time).
  // Event capacity:
  // the unattenuated per-view acceptance (d/L)^2/16 per history, 25 %
  // headroom.  Queue capacity: an isotropic photon has |d_z| below the
  // collimator's acceptance bound with probability ~w_max.  Both are rerun
  // with the exact sizes if they overflow (transport is deterministic).
  // Forced detection: chunks of 2^21 histories; the queue holds interaction
  // locations (one emission + the real collisions, ~2-3 per history), and
  // each location gives at most one weighted event per view.
  const bool forced = ts.forced != 0;
  const bool weighted = forced || ts.forced_dir != 0;
  const double band = (ts.hole_diam / ts.hole_len) / std::sqrt(1.0 + (ts.hole_diam / ts.hole_len) * (ts.hole_diam / ts.hole_len));
  const double tan_max = ts.hole_diam / ts.hole_len;
  const double w_max = tan_max / std::sqrt(1.0 + tan_max * tan_max) * 1.02 + 1e-6;
  const size_t qb = forced ? fd_rec_bytes(ts.precision) : escape_rec_bytes(ts.precision);
  uint64_t kChunk = forced ? (1ull << 21) : (1ull << 27);
  if (!forced) {
    const double q_frac = ts.forced_dir ? 1.0 : (w_max * 1.1 < 1.0 ? w_max * 1.1 : 1.0);
    while (kChunk < (1ull << 30) && (double)(2 * kChunk) * q_frac * (double)qb <= 4294967296.0) kChunk *= 2;
  }
  const uint64_t n_chunks = (count + kChunk - 1) / kChunk;
  const uint64_t chunk_max = count < kChunk ? count : kChunk;
  const double acc = tan_max * tan_max / 16.0;
  double est = forced ? (double)count * (double)ts.n_views * 2.0 + 65536.0
                      : (double)count * (double)ts.n_views * acc * 1.25 / (ts.forced_dir ? band : 1.0) + 65536.0;
  if (est > 4.0e9) est = 4.0e9;
  double est_q = forced ? (double)chunk_max * 3.0 + 65536.0
                        : (double)chunk_max * (ts.forced_dir ? 1.0 : w_max * 1.1) + 65536.0;
  if (!forced && est_q > (double)chunk_max) est_q = (double)chunk_max;
  unsigned long long cap = (unsigned long long)est, cap_q = (unsigned long long)est_q;
  DevBuf ctr, esc;
  std::vector<cudaEvent_t> evs(3 * n_chunks, nullptr);
  struct EvGuard {
    std::vector<cudaEvent_t> &v;
    ~EvGuard() { for (cudaEvent_t e : v) if (e) cudaEventDestroy(e); }
  } eg{evs};
  for (auto &e : evs)
    if (cudaEventCreate(&e) != cudaSuccess) { set_error("cudaEventCreate failed"); return MC_ECUDA; }
  MCS_TRY(ctr.alloc(kCounters * sizeof(unsigned long long), s));
  unsigned long long *hctr = out.hctr;
  for (int attempt = 0; attempt < 3; ++attempt) {
    MCS_TRY(out.events.alloc(cap * sizeof(unsigned long long), s));
    if (weighted) MCS_TRY(out.weights.alloc(cap * sizeof(unsigned long long), s));
    MCS_TRY(esc.alloc(cap_q * qb, s));
    MCS_CUDA(cudaMemsetAsync(ctr.p, 0, kCounters * sizeof(unsigned long long), s));
    ts.events = out.events.as<unsigned long long>();
    ts.capacity = cap;
    ts.cursor = ctr.as<unsigned long long>();
    ts.fates = ctr.as<unsigned long long>() + 1;
    ts.esc = esc.p;
    ts.esc_capacity = cap_q;
    ts.esc_cursor = ctr.as<unsigned long long>() + 5;
    ts.records = nullptr;
    ts.weights = weighted ? out.weights.as<unsigned long long>() : nullptr;
    for (uint64_t c = 0; c < n_chunks; ++c) {
      ts.first = first + c * kChunk;
      ts.count = (c + 1 < n_chunks) ? kChunk : count - c * kChunk;
      ts.ev_mid = evs[3 * c + 1];
      cudaEventRecord(evs[3 * c], s);
      MCS_TRY(run_transport(ts, s));
      cudaEventRecord(evs[3 * c + 2], s);
      // remember the largest queue fill, empty the queue for the next chunk
      count_launch();
      queue_reset_kernel<<<1, 1, 0, s>>>(ctr.as<unsigned long long>());
      if (cudaGetLastError() != cudaSuccess) { set_error("queue reset launch failed"); return MC_ECUDA; }
    }
    if (cudaMemcpyAsync(hctr, ctr.p, kCounters * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("transport failed: %s", cudaGetErrorString(cudaGetLastError()));
      return MC_ECUDA;
    }
    {
      // every history ends in exactly one fate; fewer means a transport
      // launch gave up (its random-word producer stopped answering)
      const unsigned long long done = hctr[1] + hctr[2] + hctr[3] + hctr[4];
      if (done != count) {
        set_error("transport finished %llu of %llu histories", done, (unsigned long long)count);
        return MC_ECUDA;
      }
    }
    if (hctr[0] <= cap && hctr[6] <= cap_q) break;
    if (hctr[0] >= 0xFFFFFFFFull) {
      set_error("%llu events exceed the 2^32 limit of one build; split the history range", hctr[0]);
      return MC_EINVAL;
    }
    // rerun with room for everything counted (a lost queue entry also lost
    // its detections, so the event count can grow once more)
    if (hctr[6] > cap_q) cap_q = hctr[6];
    if (hctr[0] > cap) cap = hctr[0] + hctr[0] / 8;
    if (attempt == 2) {
      set_error("transport buffers kept overflowing");
      return MC_ECUDA;
    }
  }
  for (uint64_t c = 0; c < n_chunks; ++c) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, evs[3 * c], evs[3 * c + 1]);
    cudaEventElapsedTime(&b, evs[3 * c + 1], evs[3 * c + 2]);
    out.ms_transport += a;
    out.ms_detect += b;
  }
  return MC_OK;
}

static int build_from_plan(mc_plan *pl, uint64_t first, uint64_t count, uint64_t seed, cudaStream_t s,
                           mc_system **out) {
  mc_system *sys = new (std::nothrow) mc_system();
  if (!sys) { set_error("out of host memory"); return MC_ENOMEM; }
  auto fail = [&](int rc) { delete sys; return rc; };
  const TransportSetup &ts = pl->ts;
  sys->n_rows = (int64_t)ts.n_views * ts.bins_u * ts.bins_v;
  sys->n_cols = (int64_t)ts.nx * ts.ny * ts.nz;
  sys->first = first;
  sys->count = count;
  const bool weighted = ts.forced != 0 || ts.forced_dir != 0;
  Tally t;
  int rc = tally_from_plan(pl, first, count, seed, s, t);
  if (rc) return fail(rc);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    set_error("cudaEventCreate failed");
    return fail(MC_ECUDA);
  }
  cudaEventRecord(e0, s);
  sys->n_events = (int64_t)t.hctr[0];
  for (int f = 0; f < 4; ++f) sys->fates[f] = t.hctr[1 + f];
  rc = assemble_system(sys, t.events, sys->n_events, s, weighted ? t.weights.as<uint64_t>() : nullptr);
  if (rc == MC_OK) {
    t.weights.release();
    rc = finish_system(sys, s);
  }
  float t_asm = 0.f;
  if (rc == MC_OK) {
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&t_asm, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return fail(rc);
  sys->ms_transport = t.ms_transport;
  sys->ms_detect = t.ms_detect;
  sys->ms_assembly = t_asm;
  *out = sys;
  return MC_OK;
}

__global__ void events_to_keys_kernel(const int32_t *rows, const int32_t *cols, int64_t n, uint64_t m,
                                      unsigned long long *keys) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    keys[i] = (unsigned long long)cols[i] * m + (unsigned long long)rows[i];
}

// ---------------------------------------------------------------------------
// routing tally events to the parts that own their views (multi-GPU split)
// ---------------------------------------------------------------------------
constexpr int kMaxParts = 1024;
constexpr int kRouteThreads = 256;

// Part of event key v M + j: part_of_view[j / rows_per_view].
__device__ __forceinline__ int route_part(uint64_t key, uint64_t m, uint64_t rpv, const int32_t *part_of_view) {
  return part_of_view[(key % m) / rpv];
}

__global__ void route_count_kernel(const uint64_t *keys, int64_t n, uint64_t m, uint64_t rpv,
                                   const int32_t *part_of_view, int n_parts, unsigned long long *counts) {
  __shared__ unsigned int s_cnt[kMaxParts];
  for (int p = threadIdx.x; p < n_parts; p += blockDim.x) s_cnt[p] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&s_cnt[route_part(keys[i], m, rpv, part_of_view)], 1u);
  __syncthreads();
  for (int p = threadIdx.x; p < n_parts; p += blockDim.x)
    if (s_cnt[p]) atomicAdd(&counts[p], (unsigned long long)s_cnt[p]);
}

// Each block handles one contiguous chunk of the keys: counts its events per
// part, reserves a range per part from the global cursors, then writes each
// event, renumbered to its part's rows (key' = v M_p + j - row0_p), into the
// part's range.  The order inside a part is not fixed; assembly sorts.
__global__ void route_scatter_kernel(const uint64_t *keys, int64_t n, uint64_t m, uint64_t rpv,
                                     const int32_t *part_of_view, const uint64_t *row0, const uint64_t *m_part,
                                     int n_parts, int64_t chunk, unsigned long long *cursor, uint64_t *out) {
  __shared__ unsigned int s_cnt[kMaxParts];
  __shared__ unsigned long long s_base[kMaxParts];
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
  for (int p = threadIdx.x; p < n_parts; p += blockDim.x) s_cnt[p] = 0u;
  __syncthreads();
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x)
    atomicAdd(&s_cnt[route_part(keys[i], m, rpv, part_of_view)], 1u);
  __syncthreads();
  for (int p = threadIdx.x; p < n_parts; p += blockDim.x) {
    s_base[p] = s_cnt[p] ? atomicAdd(&cursor[p], (unsigned long long)s_cnt[p]) : 0ull;
    s_cnt[p] = 0u;
  }
  __syncthreads();
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const uint64_t k = keys[i];
    const uint64_t j = k % m, v = k / m;
    const int p = part_of_view[j / rpv];
    const unsigned int o = atomicAdd(&s_cnt[p], 1u);
    out[s_base[p] + o] = v * m_part[p] + (j - row0[p]);
  }
}

// largest key of a list (validation of keys handed in by the caller)
__global__ void max_key_kernel(const uint64_t *keys, int64_t n, unsigned long long *mx) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = keys[i] > m ? keys[i] : m;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
    m = t > m ? t : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

}  // namespace mcs

using namespace mcs;

#define API_STREAM(x) (static_cast<cudaStream_t>(x))

extern "C" {

const char *mc_last_error(void) { return g_error.c_str(); }

uint64_t mc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int mc_plan_create(const mc_phantom *phantom, const mc_geometry *geometry, void *stream, mc_plan **out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return MC_EINVAL; }
  *out = nullptr;
  return make_plan(phantom, geometry, API_STREAM(stream), out);
}

int mc_plan_build(mc_plan *plan, uint64_t first, uint64_t count, uint64_t seed, void *stream, mc_system **out) {
  clear_error();
  if (!plan || !out) { set_error("NULL argument"); return MC_EINVAL; }
  *out = nullptr;
  return build_from_plan(plan, first, count, seed, API_STREAM(stream), out);
}

int mc_plan_tally(mc_plan *plan, uint64_t first, uint64_t count, uint64_t seed, uint64_t *keys_dev, int64_t capacity,
                  int64_t *n_events_out, uint64_t *fates_host, void *stream) {
  clear_error();
  if (!plan || !n_events_out) { set_error("NULL argument"); return MC_EINVAL; }
  if (plan->ts.forced || plan->ts.forced_dir) {
    set_error("mc_plan_tally: weighted (forced-detection / forced-direction) plans have no plain event list");
    return MC_EINVAL;
  }
  if (capacity < 0 || (capacity > 0 && !keys_dev)) { set_error("bad key buffer"); return MC_EINVAL; }
  cudaStream_t s = API_STREAM(stream);
  Tally t;
  MCS_TRY(tally_from_plan(plan, first, count, seed, s, t));
  const int64_t n = (int64_t)t.hctr[0];
  *n_events_out = n;
  if (fates_host)
    for (int f = 0; f < 4; ++f) fates_host[f] = t.hctr[1 + f];
  if (n > capacity) {
    set_error("mc_plan_tally: %lld events do not fit the buffer of %lld keys (the count is in *n_events_out; the "
              "tally is deterministic, repeat with a larger buffer)",
              (long long)n, (long long)capacity);
    return MC_EINVAL;
  }
  if (n > 0) MCS_CUDA(cudaMemcpyAsync(keys_dev, t.events.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_events_route(const uint64_t *keys_dev, int64_t n_events, int64_t n_rows, int64_t rows_per_view, int32_t n_parts,
                    uint64_t *out_dev, int64_t *part_counts_host, void *stream) {
  clear_error();
  if (!part_counts_host || (n_events > 0 && (!keys_dev || !out_dev))) { set_error("NULL argument"); return MC_EINVAL; }
  if (n_events < 0 || n_rows < 1 || rows_per_view < 1 || n_rows % rows_per_view != 0) {
    set_error("sizes out of range: n_rows must be a positive multiple of rows_per_view");
    return MC_EINVAL;
  }
  const int64_t n_views = n_rows / rows_per_view;
  if (n_parts < 1 || n_parts > kMaxParts || n_parts > n_views) {
    set_error("n_parts must be in 1 .. min(views, %d)", kMaxParts);
    return MC_EINVAL;
  }
  std::vector<int32_t> pov((size_t)n_views);
  std::vector<uint64_t> row0((size_t)n_parts), m_part((size_t)n_parts);
  for (int p = 0; p < n_parts; ++p) {
    const int64_t v0 = (int64_t)p * n_views / n_parts, v1 = (int64_t)(p + 1) * n_views / n_parts;
    for (int64_t k = v0; k < v1; ++k) pov[(size_t)k] = p;
    row0[(size_t)p] = (uint64_t)(v0 * rows_per_view);
    m_part[(size_t)p] = (uint64_t)((v1 - v0) * rows_per_view);
  }
  cudaStream_t s = API_STREAM(stream);
  DevBuf d_pov, d_row0, d_m, d_cnt;
  MCS_TRY(d_pov.alloc(pov.size() * 4, s));
  MCS_TRY(d_row0.alloc((size_t)n_parts * 8, s));
  MCS_TRY(d_m.alloc((size_t)n_parts * 8, s));
  MCS_TRY(d_cnt.alloc((size_t)n_parts * 8 * 2, s));
  MCS_CUDA(cudaMemcpyAsync(d_pov.p, pov.data(), pov.size() * 4, cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(d_row0.p, row0.data(), (size_t)n_parts * 8, cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemcpyAsync(d_m.p, m_part.data(), (size_t)n_parts * 8, cudaMemcpyHostToDevice, s));
  MCS_CUDA(cudaMemsetAsync(d_cnt.p, 0, (size_t)n_parts * 8 * 2, s));
  unsigned long long *cnt = d_cnt.as<unsigned long long>(), *cursor = cnt + n_parts;
  std::vector<unsigned long long> h((size_t)n_parts, 0ull);
  if (n_events > 0) {
    int g = (int)((n_events + kRouteThreads - 1) / kRouteThreads);
    if (g > device_sm_count() * 8) g = device_sm_count() * 8;
    count_launch();
    route_count_kernel<<<g, kRouteThreads, 0, s>>>(keys_dev, n_events, (uint64_t)n_rows, (uint64_t)rows_per_view,
                                                   d_pov.as<int32_t>(), n_parts, cnt);
    MCS_LAUNCHED();
    MCS_CUDA(cudaMemcpyAsync(h.data(), cnt, (size_t)n_parts * 8, cudaMemcpyDeviceToHost, s));
    MCS_CUDA(cudaStreamSynchronize(s));
    std::vector<unsigned long long> start((size_t)n_parts, 0ull);
    for (int p = 1; p < n_parts; ++p) start[(size_t)p] = start[(size_t)p - 1] + h[(size_t)p - 1];
    MCS_CUDA(cudaMemcpyAsync(cursor, start.data(), (size_t)n_parts * 8, cudaMemcpyHostToDevice, s));
    const int64_t chunk = 8192;
    const int64_t nb = (n_events + chunk - 1) / chunk;
    count_launch();
    route_scatter_kernel<<<(unsigned)nb, kRouteThreads, 0, s>>>(keys_dev, n_events, (uint64_t)n_rows,
                                                                (uint64_t)rows_per_view, d_pov.as<int32_t>(),
                                                                d_row0.as<uint64_t>(), d_m.as<uint64_t>(), n_parts,
                                                                chunk, cursor, out_dev);
    MCS_LAUNCHED();
  }
  MCS_CUDA(cudaStreamSynchronize(s));
  for (int p = 0; p < n_parts; ++p) part_counts_host[p] = (int64_t)h[(size_t)p];
  return MC_OK;
}

int mc_system_from_keys(int64_t n_rows, int64_t n_cols, const uint64_t *keys_dev, int64_t n_keys, uint64_t first,
                        uint64_t count, void *stream, mc_system **out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return MC_EINVAL; }
  *out = nullptr;
  if (n_rows < 1 || n_cols < 1 || n_rows >= (1ll << 31) || n_cols >= (1ll << 31) || n_keys < 0 ||
      n_keys >= 0xFFFFFFFFll) {
    set_error("sizes out of range");
    return MC_EINVAL;
  }
  if (n_keys > 0 && !keys_dev) { set_error("keys_dev is NULL"); return MC_EINVAL; }
  cudaStream_t s = API_STREAM(stream);
  mc_system *sys = new (std::nothrow) mc_system();
  if (!sys) { set_error("out of host memory"); return MC_ENOMEM; }
  auto fail = [&](int rc) { delete sys; return rc; };
  sys->n_rows = n_rows;
  sys->n_cols = n_cols;
  sys->first = first;
  sys->count = count;
  sys->n_events = n_keys;
  DevBuf keys, mx;
  int rc;
  if ((rc = keys.alloc((size_t)(n_keys > 0 ? n_keys : 1) * 8, s)) || (rc = mx.alloc(8, s))) return fail(rc);
  if (n_keys > 0) {
    if (cudaMemcpyAsync(keys.p, keys_dev, (size_t)n_keys * 8, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(mx.p, 0, 8, s) != cudaSuccess) {
      set_error("key copy failed");
      return fail(MC_ECUDA);
    }
    int g = (int)((n_keys + 255) / 256);
    if (g > device_sm_count() * 8) g = device_sm_count() * 8;
    count_launch();
    max_key_kernel<<<g, 256, 0, s>>>(keys.as<uint64_t>(), n_keys, mx.as<unsigned long long>());
    unsigned long long hmx = 0;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(&hmx, mx.p, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("key check failed");
      return fail(MC_ECUDA);
    }
    if (hmx >= (unsigned long long)n_rows * (unsigned long long)n_cols) {
      set_error("key %llu is out of range for %lld rows x %lld columns", hmx, (long long)n_rows, (long long)n_cols);
      return fail(MC_EINVAL);
    }
  }
  if ((rc = assemble_system(sys, keys, n_keys, s))) return fail(rc);
  if ((rc = finish_system(sys, s))) return fail(rc);
  *out = sys;
  return MC_OK;
}

int mc_plan_free(mc_plan *plan) {
  clear_error();
  delete plan;
  return MC_OK;
}

int mc_build_system(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t n_histories, uint64_t seed,
                    void *stream, mc_system **out) {
  return mc_build_system_range(phantom, geometry, 0, n_histories, seed, stream, out);
}

int mc_build_system_range(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t first, uint64_t count,
                          uint64_t seed, void *stream, mc_system **out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return MC_EINVAL; }
  *out = nullptr;
  mc_plan *pl = nullptr;
  MCS_TRY(make_plan(phantom, geometry, API_STREAM(stream), &pl));
  const int rc = build_from_plan(pl, first, count, seed, API_STREAM(stream), out);
  delete pl;
  return rc;
}

int mc_system_from_events(int64_t n_rows, int64_t n_cols, const int32_t *rows_host, const int32_t *cols_host,
                          int64_t n_events, uint64_t first, uint64_t count, void *stream, mc_system **out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return MC_EINVAL; }
  *out = nullptr;
  if (n_rows < 1 || n_cols < 1 || n_rows >= (1ll << 31) || n_cols >= (1ll << 31) || n_events < 0 ||
      n_events >= 0xFFFFFFFFll) {
    set_error("sizes out of range");
    return MC_EINVAL;
  }
  if (n_events > 0 && (!rows_host || !cols_host)) { set_error("event arrays are NULL"); return MC_EINVAL; }
  for (int64_t i = 0; i < n_events; ++i) {
    if (rows_host[i] < 0 || rows_host[i] >= n_rows || cols_host[i] < 0 || cols_host[i] >= n_cols) {
      set_error("event %lld (%d, %d) out of range", (long long)i, rows_host[i], cols_host[i]);
      return MC_EINVAL;
    }
  }
  cudaStream_t s = API_STREAM(stream);
  mc_system *sys = new (std::nothrow) mc_system();
  if (!sys) { set_error("out of host memory"); return MC_ENOMEM; }
  auto fail = [&](int rc) { delete sys; return rc; };
  sys->n_rows = n_rows;
  sys->n_cols = n_cols;
  sys->first = first;
  sys->count = count;
  sys->n_events = n_events;
  DevBuf keys, r, c;
  int rc;
  const size_t nb = (size_t)(n_events > 0 ? n_events : 1);
  if ((rc = keys.alloc(nb * 8, s)) || (rc = r.alloc(nb * 4, s)) || (rc = c.alloc(nb * 4, s))) return fail(rc);
  if (n_events > 0) {
    if (cudaMemcpyAsync(r.p, rows_host, n_events * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c.p, cols_host, n_events * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("event upload failed");
      return fail(MC_ECUDA);
    }
    int g = (int)((n_events + 255) / 256);
    if (g > 65535) g = 65535;
    count_launch(); events_to_keys_kernel<<<g, 256, 0, s>>>(r.as<int32_t>(), c.as<int32_t>(), n_events, (uint64_t)n_rows,
                                            keys.as<unsigned long long>());
    if (cudaGetLastError() != cudaSuccess) { set_error("key kernel launch failed"); return fail(MC_ECUDA); }
  }
  r.release();
  c.release();
  if ((rc = assemble_system(sys, keys, n_events, s))) return fail(rc);
  if ((rc = finish_system(sys, s))) return fail(rc);
  *out = sys;
  return MC_OK;
}

int mc_system_from_weighted_events(int64_t n_rows, int64_t n_cols, const int32_t *rows_host, const int32_t *cols_host,
                                   const uint64_t *weights_host, int64_t n_events, uint64_t first, uint64_t count,
                                   void *stream, mc_system **out) {
  clear_error();
  if (!out) { set_error("out is NULL"); return MC_EINVAL; }
  *out = nullptr;
  if (n_rows < 1 || n_cols < 1 || n_rows >= (1ll << 31) || n_cols >= (1ll << 31) || n_events < 0 ||
      n_events >= 0xFFFFFFFFll) {
    set_error("sizes out of range");
    return MC_EINVAL;
  }
  if (n_events > 0 && (!rows_host || !cols_host || !weights_host)) { set_error("event arrays are NULL"); return MC_EINVAL; }
  for (int64_t i = 0; i < n_events; ++i) {
    if (rows_host[i] < 0 || rows_host[i] >= n_rows || cols_host[i] < 0 || cols_host[i] >= n_cols) {
      set_error("event %lld (%d, %d) out of range", (long long)i, rows_host[i], cols_host[i]);
      return MC_EINVAL;
    }
  }
  cudaStream_t s = API_STREAM(stream);
  mc_system *sys = new (std::nothrow) mc_system();
  if (!sys) { set_error("out of host memory"); return MC_ENOMEM; }
  auto fail = [&](int rc) { delete sys; return rc; };
  sys->n_rows = n_rows;
  sys->n_cols = n_cols;
  sys->first = first;
  sys->count = count;
  sys->n_events = n_events;
  DevBuf keys, r, c, w;
  int rc;
  const size_t nb = (size_t)(n_events > 0 ? n_events : 1);
  if ((rc = keys.alloc(nb * 8, s)) || (rc = r.alloc(nb * 4, s)) || (rc = c.alloc(nb * 4, s)) ||
      (rc = w.alloc(nb * 8, s)))
    return fail(rc);
  if (n_events > 0) {
    if (cudaMemcpyAsync(r.p, rows_host, n_events * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c.p, cols_host, n_events * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(w.p, weights_host, n_events * 8, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("event upload failed");
      return fail(MC_ECUDA);
    }
    int g = (int)((n_events + 255) / 256);
    if (g > 65535) g = 65535;
    count_launch(); events_to_keys_kernel<<<g, 256, 0, s>>>(r.as<int32_t>(), c.as<int32_t>(), n_events, (uint64_t)n_rows,
                                            keys.as<unsigned long long>());
    if (cudaGetLastError() != cudaSuccess) { set_error("key kernel launch failed"); return fail(MC_ECUDA); }
  }
  r.release();
  c.release();
  if ((rc = assemble_system(sys, keys, n_events, s, w.as<uint64_t>()))) return fail(rc);
  w.release();
  if ((rc = finish_system(sys, s))) return fail(rc);
  *out = sys;
  return MC_OK;
}

__global__ void entries_to_f64_kernel(const uint32_t *cnt, const uint64_t *wq, int64_t n, double *out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = wq ? (double)wq[i] * (1.0 / kFdScale) : (double)cnt[i];
}

int mc_system_export_values(const mc_system *sys, double *csc_values_host, double *csr_values_host, void *stream) {
  clear_error();
  if (!sys) { set_error("system is NULL"); return MC_EINVAL; }
  if (sys->nnz == 0) return MC_OK;
  cudaStream_t s = API_STREAM(stream);
  DevBuf tmp;
  MCS_TRY(tmp.alloc((size_t)sys->nnz * sizeof(double), s));
  int g = (int)((sys->nnz + 255) / 256);
  if (g > 65535) g = 65535;
  for (int side = 0; side < 2; ++side) {
    double *dst = side == 0 ? csc_values_host : csr_values_host;
    if (!dst) continue;
    const DevBuf &cnt = side == 0 ? sys->csc_cnt : sys->csr_cnt;
    const DevBuf &wq = side == 0 ? sys->csc_wq : sys->csr_wq;
    count_launch();
    entries_to_f64_kernel<<<g, 256, 0, s>>>(cnt.as<uint32_t>(), sys->weighted ? wq.as<uint64_t>() : nullptr, sys->nnz,
                                            tmp.as<double>());
    MCS_CUDA(cudaGetLastError());
    MCS_CUDA(cudaMemcpyAsync(dst, tmp.p, (size_t)sys->nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_system_free(mc_system *sys) {
  clear_error();
  if (!sys) return MC_OK;
  delete sys;  // DevBufs release their memory on their own streams
  return MC_OK;
}

int mc_system_info_get(const mc_system *sys, mc_system_info *info) {
  clear_error();
  if (!sys || !info) { set_error("NULL argument"); return MC_EINVAL; }
  info->n_rows = sys->n_rows;
  info->n_cols = sys->n_cols;
  info->nnz = sys->nnz;
  info->n_events = sys->n_events;
  info->first_history = sys->first;
  info->n_histories = sys->count;
  for (int f = 0; f < 4; ++f) info->fates[f] = sys->fates[f];
  info->max_count = sys->max_count;
  info->value_type = sys->value_type;
  info->build_ms_transport = sys->ms_transport;
  info->build_ms_assembly = sys->ms_assembly;
  info->build_ms_detect = sys->ms_detect;
  info->spmv_fwd = sys->n_csr_blocks > 0 ? 0 : sys->spmv_group_fwd;
  info->spmv_bwd = sys->n_csc_blocks > 0 ? 0 : sys->spmv_group_bwd;
  info->weighted = sys->weighted ? 1 : 0;
  return MC_OK;
}

static int copy_ptr_u32_to_i64(const DevBuf &src, int64_t n, int64_t *dst, cudaStream_t s) {
  std::vector<uint32_t> tmp((size_t)n);
  MCS_CUDA(cudaMemcpyAsync(tmp.data(), src.p, n * 4, cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; ++i) dst[i] = tmp[i];
  return MC_OK;
}

int mc_system_export_csc(const mc_system *sys, int64_t *col_ptr_host, int32_t *row_idx_host, uint32_t *counts_host,
                         uint32_t *n_v_host, void *stream) {
  clear_error();
  if (!sys) { set_error("system is NULL"); return MC_EINVAL; }
  cudaStream_t s = API_STREAM(stream);
  if (col_ptr_host) MCS_TRY(copy_ptr_u32_to_i64(sys->col_ptr, sys->n_cols + 1, col_ptr_host, s));
  if (row_idx_host && sys->nnz) MCS_CUDA(cudaMemcpyAsync(row_idx_host, sys->row_idx.p, sys->nnz * 4, cudaMemcpyDeviceToHost, s));
  if (counts_host && sys->nnz) MCS_CUDA(cudaMemcpyAsync(counts_host, sys->csc_cnt.p, sys->nnz * 4, cudaMemcpyDeviceToHost, s));
  if (n_v_host) MCS_CUDA(cudaMemcpyAsync(n_v_host, sys->n_v.p, sys->n_cols * 4, cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_system_export_csr(const mc_system *sys, int64_t *row_ptr_host, int32_t *col_idx_host, uint32_t *counts_host,
                         void *stream) {
  clear_error();
  if (!sys) { set_error("system is NULL"); return MC_EINVAL; }
  cudaStream_t s = API_STREAM(stream);
  if (row_ptr_host) MCS_TRY(copy_ptr_u32_to_i64(sys->row_ptr, sys->n_rows + 1, row_ptr_host, s));
  if (col_idx_host && sys->nnz) MCS_CUDA(cudaMemcpyAsync(col_idx_host, sys->col_idx.p, sys->nnz * 4, cudaMemcpyDeviceToHost, s));
  if (counts_host && sys->nnz) MCS_CUDA(cudaMemcpyAsync(counts_host, sys->csr_cnt.p, sys->nnz * 4, cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_system_set_value_type(mc_system *sys, int32_t value_type, int32_t allow_rounding) {
  clear_error();
  if (!sys) { set_error("system is NULL"); return MC_EINVAL; }
  if (value_type != MC_VAL_F32 && value_type != MC_VAL_F16 && value_type != MC_VAL_BF16 &&
      value_type != MC_VAL_F16_A && value_type != MC_VAL_BF16_A) {
    set_error("unknown value type %d", value_type);
    return MC_EINVAL;
  }
  const uint32_t exact = value_type == MC_VAL_F32 ? (1u << 24) : value_type == MC_VAL_F16 ? 2048u : 256u;
  if (!values_are_a(value_type) && !allow_rounding && sys->max_count > exact) {
    set_error("largest count %u is not exact in the requested type (limit %u)", sys->max_count, exact);
    return MC_EINVAL;
  }
  const int old = sys->value_type;
  sys->value_type = value_type;
  cudaStream_t s = nullptr;
  int rc = make_values(sys, s);
  if (rc == MC_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = MC_ECUDA;
  if (rc != MC_OK) {
    sys->value_type = old;
    make_values(sys, s);
    cudaStreamSynchronize(s);
  }
  return rc;
}

int mc_project(const mc_system *sys, const float *x_dev, float *q_dev, void *stream) {
  clear_error();
  if (!sys || !x_dev || !q_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return project(sys, x_dev, q_dev, API_STREAM(stream));
}

int mc_backproject(const mc_system *sys, const float *r_dev, float *b_dev, void *stream) {
  clear_error();
  if (!sys || !r_dev || !b_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return backproject(sys, r_dev, b_dev, API_STREAM(stream));
}

int mc_sensitivity(const mc_system *sys, double *s_dev, void *stream) {
  clear_error();
  if (!sys || !s_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return sensitivity(sys, s_dev, API_STREAM(stream));
}

int mc_mlem_init(mc_system *sys, const float *y_dev, float *x_dev, void *stream) {
  clear_error();
  if (!sys || !y_dev || !x_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return mlem_init(sys, y_dev, x_dev, API_STREAM(stream));
}

int mlem_iterate(mc_system *sys, const float *y_dev, float *x_dev, int32_t n_iter, double *loglik_host,
                 void *stream) {
  clear_error();
  if (!sys || !y_dev || !x_dev) { set_error("NULL argument"); return MC_EINVAL; }
  if (n_iter < 0) { set_error("n_iter must be >= 0"); return MC_EINVAL; }
  cudaStream_t s = API_STREAM(stream);
  const bool want = loglik_host != nullptr && n_iter > 0;
  if (want && sys->ll_cap < n_iter) {
    MCS_TRY(sys->ll.alloc((size_t)n_iter * sizeof(double), s));
    sys->ll_cap = n_iter;
  }
  MCS_TRY(mlem_run(sys, y_dev, x_dev, n_iter, want, s));
  if (want) {
    MCS_CUDA(cudaMemcpyAsync(loglik_host, sys->ll.p, (size_t)n_iter * sizeof(double), cudaMemcpyDeviceToHost, s));
    MCS_CUDA(cudaStreamSynchronize(s));
  }
  return MC_OK;
}

int mc_system_subset(const mc_system *parent, int64_t rows_per_view, int32_t n_subsets, int32_t subset, void *stream,
                     mc_system **out) {
  clear_error();
  if (!parent || !out) { set_error("NULL argument"); return MC_EINVAL; }
  *out = nullptr;
  if (parent->row_map.p) { set_error("the parent is itself a subset"); return MC_EINVAL; }
  if (parent->weighted) { set_error("ordered subsets of weighted (forced-detection) systems are not supported"); return MC_EINVAL; }
  if (rows_per_view < 1 || parent->n_rows % rows_per_view != 0) {
    set_error("rows_per_view must divide the %lld rows", (long long)parent->n_rows);
    return MC_EINVAL;
  }
  const int64_t V = parent->n_rows / rows_per_view;
  if (n_subsets < 1 || n_subsets > V || subset < 0 || subset >= n_subsets) {
    set_error("need 1 <= n_subsets <= %lld views and 0 <= subset < n_subsets", (long long)V);
    return MC_EINVAL;
  }
  cudaStream_t s = API_STREAM(stream);
  mc_system *sys = new (std::nothrow) mc_system();
  if (!sys) { set_error("out of host memory"); return MC_ENOMEM; }
  int rc = subset_system(parent, rows_per_view, n_subsets, subset, sys, s);
  if (rc == MC_OK) rc = finish_system(sys, s);
  if (rc != MC_OK) { delete sys; return rc; }
  *out = sys;
  return MC_OK;
}

int osem_iterate(mc_system *const *fwd, mc_system *const *back, int32_t n_subsets, const float *y_dev,
                 const float *add_dev, float *x_dev, int32_t n_iter, void *stream) {
  clear_error();
  if (!fwd || !back || !y_dev || !x_dev) { set_error("NULL argument"); return MC_EINVAL; }
  if (n_subsets < 1 || n_iter < 0) { set_error("n_subsets must be >= 1 and n_iter >= 0"); return MC_EINVAL; }
  for (int k = 0; k < n_subsets; ++k) {
    const mc_system *f = fwd[k], *b = back[k];
    if (!f || !b) { set_error("subset %d: NULL system", k); return MC_EINVAL; }
    if (f->n_subsets != n_subsets || b->n_subsets != n_subsets || f->subset != k || b->subset != k) {
      set_error("subset %d: systems must be subset %d of %d (got %d of %d and %d of %d)", k, k, n_subsets, f->subset,
                f->n_subsets, b->subset, b->n_subsets);
      return MC_EINVAL;
    }
    if (f->n_rows != b->n_rows || f->n_cols != b->n_cols || f->parent_rows != fwd[0]->parent_rows ||
        b->parent_rows != fwd[0]->parent_rows || f->n_cols != fwd[0]->n_cols) {
      set_error("subset %d: forward and back-projection systems differ in shape", k);
      return MC_EINVAL;
    }
  }
  return osem_run(fwd, back, n_subsets, y_dev, add_dev, x_dev, n_iter, API_STREAM(stream));
}

int mc_project_ratio(const mc_system *sys, const float *x_dev, const float *y_dev, float *r_dev, void *stream) {
  clear_error();
  if (!sys || !x_dev || !y_dev || !r_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return project_ratio(sys, x_dev, y_dev, r_dev, API_STREAM(stream));
}

int mc_loglik(const mc_system *sys, const float *x_dev, const float *y_dev, double *value_dev, void *stream) {
  clear_error();
  if (!sys || !x_dev || !y_dev || !value_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return loglik(sys, x_dev, y_dev, value_dev, API_STREAM(stream));
}

int mc_project_f64(const mc_system *sys, const double *x_dev, double *q_dev, void *stream) {
  clear_error();
  if (!sys || !x_dev || !q_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return project_f64(sys, x_dev, q_dev, API_STREAM(stream));
}

int mc_backproject_f64(const mc_system *sys, const double *r_dev, double *b_dev, void *stream) {
  clear_error();
  if (!sys || !r_dev || !b_dev) { set_error("NULL argument"); return MC_EINVAL; }
  return backproject_f64(sys, r_dev, b_dev, API_STREAM(stream));
}

static int check_prior(int32_t nx, int32_t ny, int32_t nz, double beta, const void *x) {
  if (!x) { set_error("x is NULL"); return MC_EINVAL; }
  if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= (1ll << 40)) { set_error("bad grid"); return MC_EINVAL; }
  if (!(beta >= 0.0) || !std::isfinite(beta)) { set_error("beta must be finite and >= 0"); return MC_EINVAL; }
  return MC_OK;
}

int mc_prior_quadratic(int32_t nx, int32_t ny, int32_t nz, double beta, const float *x_dev, float *grad_dev,
                       double *value_dev, void *stream) {
  clear_error();
  MCS_TRY(check_prior(nx, ny, nz, beta, x_dev));
  return prior_quadratic<float>(nx, ny, nz, beta, x_dev, grad_dev, value_dev, API_STREAM(stream));
}

int mc_prior_quadratic_f64(int32_t nx, int32_t ny, int32_t nz, double beta, const double *x_dev, double *grad_dev,
                           double *value_dev, void *stream) {
  clear_error();
  MCS_TRY(check_prior(nx, ny, nz, beta, x_dev));
  return prior_quadratic<double>(nx, ny, nz, beta, x_dev, grad_dev, value_dev, API_STREAM(stream));
}

int mc_pgd_step(int64_t n, double alpha, const double *sens_dev, const float *bp_dev, const float *gp_dev,
                float *x_dev, void *stream) {
  clear_error();
  if (!sens_dev || !bp_dev || !x_dev || n < 0) { set_error("NULL argument or negative size"); return MC_EINVAL; }
  if (!(alpha > 0.0) || !std::isfinite(alpha)) { set_error("alpha must be positive"); return MC_EINVAL; }
  return pgd_step(n, alpha, sens_dev, bp_dev, gp_dev, x_dev, API_STREAM(stream));
}

int mc_vector_sum(int64_t n, const float *v_dev, double *out_dev, void *stream) {
  clear_error();
  if (n < 0 || !out_dev || (n > 0 && !v_dev)) { set_error("bad argument"); return MC_EINVAL; }
  return vector_sum(n, v_dev, out_dev, API_STREAM(stream));
}

int mc_mlem_start(int64_t n, const double *sens_dev, double sum_y, float *x_dev, void *stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!sens_dev || !x_dev))) { set_error("bad argument"); return MC_EINVAL; }
  return mlem_start(n, sens_dev, sum_y, x_dev, API_STREAM(stream));
}

int mc_system_set_spmv_layout(mc_system *sys, int32_t fwd, int32_t bwd, void *stream) {
  clear_error();
  if (!sys) { set_error("system is NULL"); return MC_EINVAL; }
  return set_spmv_layout(sys, fwd, bwd, API_STREAM(stream));
}

int mc_system_autotune(mc_system *sys, void *stream) {
  clear_error();
  if (!sys) { set_error("system is NULL"); return MC_EINVAL; }
  int f = 0, b = 0;
  return autotune(sys, API_STREAM(stream), &f, &b);
}

int mc_batch_create(mc_system *const *systems, int32_t n, const float *const *y_dev, float *const *x_dev,
                    mc_batch **out) {
  clear_error();
  if (!systems || !y_dev || !x_dev || !out || n < 1) { set_error("NULL argument or empty batch"); return MC_EINVAL; }
  *out = nullptr;
  return batch_create(systems, n, y_dev, x_dev, out);
}

int mc_batch_mlem(mc_batch *batch, int32_t n_iter, void *stream) {
  clear_error();
  if (!batch || n_iter < 0) { set_error("NULL batch or negative n_iter"); return MC_EINVAL; }
  return batch_mlem(batch, n_iter, API_STREAM(stream));
}

int mc_batch_mlem_persistent(mc_batch *batch, int32_t n_iter, void *stream) {
  clear_error();
  if (!batch || n_iter < 0) { set_error("NULL batch or negative n_iter"); return MC_EINVAL; }
  return batch_mlem_persistent(batch, n_iter, API_STREAM(stream));
}

int mc_batch_free(mc_batch *batch) {
  clear_error();
  batch_free(batch);
  return MC_OK;
}

int mc_trace_histories(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t seed, uint64_t first,
                       uint64_t count, mc_history_record *out_host) {
  clear_error();
  MCS_TRY(check_phantom(phantom));
  MCS_TRY(check_geometry(geometry, phantom));
  if (count > 0 && !out_host) { set_error("out_host is NULL"); return MC_EINVAL; }
  if (geometry->tally & MC_TALLY_FORCED) { set_error("per-history traces are analog only (no MC_TALLY_FORCED)"); return MC_EINVAL; }
  if (count == 0) return MC_OK;
  cudaStream_t s = nullptr;
  mc_plan pl;
  MCS_TRY(prepare_plan(phantom, geometry, s, pl));
  TransportSetup ts = pl.ts;
  ts.first = first;
  ts.count = count;
  ts.key0 = (uint32_t)seed;
  ts.key1 = (uint32_t)(seed >> 32);
  DevBuf rec, ctr;
  MCS_TRY(rec.alloc(count * sizeof(mc_history_record), s));
  MCS_TRY(ctr.alloc(6 * sizeof(unsigned long long), s));
  ts.events = nullptr;
  ts.capacity = 0;
  ts.cursor = ctr.as<unsigned long long>();
  ts.fates = ctr.as<unsigned long long>() + 1;
  ts.records = rec.as<mc_history_record>();
  DevBuf esc;
  MCS_TRY(esc.alloc(count * escape_rec_bytes(ts.precision), s));
  MCS_CUDA(cudaMemsetAsync(ctr.p, 0, 6 * sizeof(unsigned long long), s));
  ts.esc = esc.p;
  ts.esc_capacity = count;
  ts.esc_cursor = ctr.as<unsigned long long>() + 5;
  ts.ev_mid = nullptr;
  MCS_TRY(run_transport(ts, s));
  MCS_CUDA(cudaMemcpyAsync(out_host, rec.p, count * sizeof(mc_history_record), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_debug_kn(double e_kev, int32_t precision, uint64_t seed, uint64_t n, double *cos_out_host,
                double *eps_out_host) {
  clear_error();
  if (n > 0 && (!cos_out_host || !eps_out_host)) { set_error("NULL output"); return MC_EINVAL; }
  if (!(e_kev > 0) || (precision != MC_FP32 && precision != MC_FP64)) { set_error("bad energy or precision"); return MC_EINVAL; }
  if (n == 0) return MC_OK;
  cudaStream_t s = nullptr;
  DevBuf c, e;
  MCS_TRY(c.alloc(n * sizeof(double), s));
  MCS_TRY(e.alloc(n * sizeof(double), s));
  if (precision == MC_FP64) MCS_TRY(launch_debug_kn_f64(e_kev, seed, n, c.as<double>(), e.as<double>(), s));
  else MCS_TRY(launch_debug_kn_f32(e_kev, seed, n, c.as<double>(), e.as<double>(), s));
  MCS_CUDA(cudaMemcpyAsync(cos_out_host, c.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaMemcpyAsync(eps_out_host, e.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

int mc_debug_beam(const mc_phantom *phantom, const mc_geometry *geometry, uint64_t seed, uint64_t n,
                  const double *p0_host, const double *d_host, double e_kev, uint64_t *through_host) {
  clear_error();
  MCS_TRY(check_phantom(phantom));
  MCS_TRY(check_geometry(geometry, phantom));
  if (!p0_host || !d_host || !through_host) { set_error("NULL argument"); return MC_EINVAL; }
  cudaStream_t s = nullptr;
  mc_plan pl;
  MCS_TRY(prepare_plan(phantom, geometry, s, pl));
  TransportSetup ts = pl.ts;
  ts.first = 0;
  ts.count = n;
  ts.key0 = (uint32_t)seed;
  ts.key1 = (uint32_t)(seed >> 32);
  DevBuf t;
  MCS_TRY(t.alloc(sizeof(unsigned long long), s));
  MCS_CUDA(cudaMemsetAsync(t.p, 0, sizeof(unsigned long long), s));
  if (geometry->precision == MC_FP64)
    MCS_TRY(launch_debug_beam_f64(ts, n, p0_host, d_host, e_kev, t.as<unsigned long long>(), s));
  else
    MCS_TRY(launch_debug_beam_f32(ts, n, p0_host, d_host, e_kev, t.as<unsigned long long>(), s));
  unsigned long long h = 0;
  MCS_CUDA(cudaMemcpyAsync(&h, t.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  *through_host = h;
  return MC_OK;
}

int mc_debug_distance_map(const mc_phantom *phantom, uint8_t *out_host) {
  clear_error();
  MCS_TRY(check_phantom(phantom));
  if (!out_host) { set_error("NULL output"); return MC_EINVAL; }
  cudaStream_t s = nullptr;
  const size_t nv = (size_t)phantom->nx * phantom->ny * phantom->nz;
  DevBuf mat, map;
  MCS_TRY(mat.alloc(nv, s));
  MCS_TRY(map.alloc(nv, s));
  MCS_CUDA(cudaMemcpyAsync(mat.p, phantom->material_host, nv, cudaMemcpyHostToDevice, s));
  MCS_TRY(build_skip_map(mat.as<uint8_t>(), phantom->nx, phantom->ny, phantom->nz, map.as<uint8_t>(), s));
  MCS_CUDA(cudaMemcpyAsync(out_host, map.p, nv, cudaMemcpyDeviceToHost, s));
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

}  // extern "C"
