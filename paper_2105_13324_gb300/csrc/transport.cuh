// transport.cuh -- persistent photon-history kernel (paper Sec. 2: follow
// each source photon until it is absorbed, leaves the energy window or
// escapes, sampling every step from the cross-sections; Sec. 3: parallel-hole
// collimation and the detection window; Sec. 5.1: the detections estimate the
// response matrix T_ij of Eq. (IMC)).
//
// Included by transport_f32.cu (production, float) and transport_f64.cu
// (verification, double, compiled with --fmad=false so that every product and
// sum is rounded as written and the per-history trace can be compared with a
// double-precision reference).
//
// One thread follows one history at a time; when its history ends it starts
// the next one of its grid-stride sequence (lane refill), so the warps stay
// full until the last histories of the launch.  Each loop iteration is one
// Woodcock flight.
#pragma once

#include <cooperative_groups.h>

#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace mcs {

namespace cg = cooperative_groups;

constexpr uint32_t kStepCap = 1000000u;   // flights per history
constexpr uint32_t kTrialCap = 10000u;    // rejection trials per scatter
constexpr double kMec2 = 510.99895;       // electron rest energy, keV
constexpr double kRe = 2.8179403262e-13;  // classical electron radius, cm
constexpr double kPi = 3.14159265358979323846;

template <typename T> struct TArgs {
  const uint8_t *mat;
  const T *coef;     // per material: double {0.1 rho, N_A Z/A, k Z^4}; float {0.1 rho N_A Z/A, 0.1 rho k Z^4}
  const T *view_cs;  // [2V] cos, sin of theta_k
  int nx, ny, nz, n_mat;
  T h, hx, hy, hz;   // voxel size, half extents
  T mu_maj, e0, e_low;
  T ratio;           // L / d
  T w_max;           // |d_z| bound above which no view can accept (with margin)
  T start_deg, inv_delta, psi_views;  // azimuth window of candidate views
  int views_per_turn;                 // 360 / delta if integral, else 0
  T sigma, plane, bin, half_bu, half_bv;
  int n_views, bins_u, bins_v;
  uint32_t n_vox;
  uint64_t n_rows;
  uint64_t first, count;
  uint32_t key0, key1;
  unsigned long long *events;
  unsigned long long capacity;
  unsigned long long *cursor;
  unsigned long long *fates;
  mc_history_record *records;
};

// Klein-Nishina total cross-section per electron, cm^2, in the order
// 2 pi re re ((1+a)/(a a) (2(1+a)/t - l/a) + l/(2a) - (1+3a)/(t t)),
// a = E/mc^2, t = 1 + 2a, l = ln t.
template <typename T> __device__ __forceinline__ T sigma_kn(T e) {
  const T a = e / (T)kMec2;
  const T t = (T)1 + (T)2 * a;
  const T l = log(t);
  const T term1 = ((T)1 + a) / (a * a) * ((T)2 * ((T)1 + a) / t - l / a);
  const T term2 = l / ((T)2 * a);
  const T term3 = ((T)1 + (T)3 * a) / (t * t);
  return (T)(2.0 * kPi) * (T)kRe * (T)kRe * (term1 + term2 - term3);
}

template <typename T> struct Energy {
  T e, sig, e3, ie3;
  __device__ __forceinline__ void set(T v) {
    e = v;
    sig = sigma_kn<T>(v);
    e3 = v * v * v;
    if constexpr (std::is_same<T, float>::value) ie3 = 1.0f / e3;
  }
};

// mu(m, E) and mu_photo(m, E) in 1/mm.
template <typename T>
__device__ __forceinline__ T mu_total(const T *c0, const T *c1, const T *c2, int m, const Energy<T> &en) {
  if constexpr (std::is_same<T, double>::value) {
    return c0[m] * (c1[m] * en.sig + c2[m] / en.e3);
  } else {
    return c0[m] * en.sig + c1[m] * en.ie3;
  }
}
template <typename T>
__device__ __forceinline__ T mu_photo(const T *c0, const T *c1, const T *c2, int m, const Energy<T> &en) {
  if constexpr (std::is_same<T, double>::value) {
    return c0[m] * (c2[m] / en.e3);
  } else {
    return c1[m] * en.ie3;
  }
}

template <typename T> __device__ __forceinline__ T neg_log(T u) {
  if constexpr (std::is_same<T, double>::value) return -log(u);
  else return -__logf(u);
}

// cos and sin of phi = 2 pi u.
template <typename T> __device__ __forceinline__ void cos_sin_2pi(T u, T &c, T &s) {
  if constexpr (std::is_same<T, double>::value) {
    const double phi = (2.0 * kPi) * u;
    c = cos(phi);
    s = sin(phi);
  } else {
    // phi - pi lies in (-pi, pi), where the fast intrinsic is accurate;
    // cos(phi) = -cos(phi - pi), sin(phi) = -sin(phi - pi).
    float sp, cp;
    __sincosf(fmaf(u, 6.28318530717958648f, -3.14159265358979324f), &sp, &cp);
    c = -cp;
    s = -sp;
  }
}

template <typename T> __device__ __forceinline__ T voxel_index(T x, T half, T h, int n) {
  T f = floor((x + half) / h);
  return f > (T)(n - 1) ? (T)(n - 1) : f;
}

// Compton scatter by rejection: mu uniform in [-1,1], eps = 1/(1 + a(1-mu)),
// accepted with probability eps^2 (eps + 1/eps - (1 - mu^2)) / 2 (the
// Klein-Nishina density over its maximum).
template <typename T> __device__ __forceinline__ bool compton(Stream &st, T e, T &mu_out, T &eps_out) {
  const T alpha = e / (T)kMec2;
  for (uint32_t t = 0; t < kTrialCap; ++t) {
    const T mu = (T)2 * uniform<T>(st.word()) - (T)1;
    const T den = (T)1 + alpha * ((T)1 - mu);
    T eps, f;
    if constexpr (std::is_same<T, double>::value) {
      eps = 1.0 / den;
      f = 0.5 * eps * eps * (eps + 1.0 / eps - (1.0 - mu * mu));
    } else {
      eps = __frcp_rn(den);
      f = 0.5f * eps * eps * (eps + den - (1.0f - mu * mu));
    }
    if (uniform<T>(st.word()) < f) {
      mu_out = mu;
      eps_out = eps;
      return true;
    }
  }
  return false;
}

// Turn direction d by polar cosine mu and azimuth phi about itself.
template <typename T> __device__ __forceinline__ void rotate(T &u, T &v, T &w, T mu, T cp, T sp) {
  const T st = sqrt(fmax((T)0, (T)1 - mu * mu));
  T nu, nv, nw;
  if (fabs(w) < (T)0.99999) {
    const T r = sqrt((T)1 - w * w);
    nu = mu * u + st * (u * w * cp - v * sp) / r;
    nv = mu * v + st * (v * w * cp + u * sp) / r;
    nw = mu * w - st * cp * r;
  } else {
    nu = st * cp;
    nv = st * sp;
    nw = (w >= (T)0 ? mu : -mu);
  }
  const T n = sqrt(nu * nu + nv * nv + nw * nw);
  u = nu / n;
  v = nv / n;
  w = nw / n;
}

struct EventSink {
  unsigned long long *events, *cursor;
  unsigned long long capacity;
  mc_history_record *rec;  // trace mode
};

__device__ __forceinline__ void push_event(const EventSink &s, unsigned long long key) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(s.cursor, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  const unsigned long long idx = base + g.thread_rank();
  if (idx < s.capacity) s.events[idx] = key;
}

// Offer view k to an escaping photon at p (inside the grid) moving along d.
template <typename T, bool TRACE>
__device__ __forceinline__ void try_view(const TArgs<T> &a, Stream &st, int k, T px, T py, T pz, T dx, T dy,
                                         T dz, uint32_t v, const EventSink &sink) {
  const T ck = a.view_cs[2 * k], sk = a.view_cs[2 * k + 1];
  const T c = dx * ck + dy * sk;
  if (!(c > (T)0)) return;
  const T stt = sqrt(fmax((T)0, (T)1 - c * c));
  if (!(a.ratio * stt < c)) return;
  const T x = a.ratio * stt / c;
  const T pass = (T)(2.0 / kPi) * (acos(x) - x * sqrt((T)1 - x * x));
  if (!(uniform<T>(st.word()) < pass)) return;
  const T t = (a.plane - (px * ck + py * sk)) / c;
  const T qx = px + t * dx, qy = py + t * dy, qz = pz + t * dz;
  T au = -qx * sk + qy * ck;
  T bv = qz;
  const T u1 = uniform<T>(st.word());
  const T u2 = uniform<T>(st.word());
  const T r = sqrt((T)2 * neg_log<T>(u1));
  T cb, sb;
  cos_sin_2pi<T>(u2, cb, sb);
  au += a.sigma * (r * cb);
  bv += a.sigma * (r * sb);
  const T fu = floor(au / a.bin + a.half_bu);
  const T fv = floor(bv / a.bin + a.half_bv);
  if (!(fu >= (T)0 && fu < (T)a.bins_u && fv >= (T)0 && fv < (T)a.bins_v)) return;
  const int64_t row = ((int64_t)k * a.bins_v + (int64_t)fv) * a.bins_u + (int64_t)fu;
  if (TRACE) {
    mc_history_record *rc = sink.rec;
    if (rc->n_events < 4) rc->event_row[rc->n_events] = (int32_t)row;
    if (rc->n_events < 255) rc->n_events += 1;
  } else {
    push_event(sink, (unsigned long long)v * a.n_rows + (unsigned long long)row);
  }
}

__device__ __forceinline__ int floor_div(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// All views in ascending order; views that cannot accept are skipped by an
// azimuth window when the views tile the full turn evenly.  The window is
// wider than the acceptance cone (a candidate needs |azimuth - theta_k| below
// the cone's half-angle), so exactly the same views are tested as in a plain
// loop, in the same order.
template <typename T, bool TRACE>
__device__ void detect(const TArgs<T> &a, Stream &st, T px, T py, T pz, T dx, T dy, T dz, uint32_t v,
                       const EventSink &sink) {
  if (!(fabs(dz) < a.w_max)) return;
  const int K = a.views_per_turn;
  if (K > 0) {
    const T phi_deg = atan2(dy, dx) * (T)(180.0 / kPi);
    const T rel = (phi_deg - a.start_deg) * a.inv_delta;
    int kmin = (int)floor(rel - a.psi_views) - 1;
    int kmax = (int)ceil(rel + a.psi_views) + 1;
    if (kmax - kmin + 1 < K) {
      const int sh = floor_div(kmin, K) * K;
      kmin -= sh;
      kmax -= sh;
      if (kmax >= K) {
        for (int k = 0; k <= kmax - K && k < a.n_views; ++k) try_view<T, TRACE>(a, st, k, px, py, pz, dx, dy, dz, v, sink);
      }
      const int hi = kmax < K - 1 ? kmax : K - 1;
      for (int k = kmin; k <= hi && k < a.n_views; ++k) try_view<T, TRACE>(a, st, k, px, py, pz, dx, dy, dz, v, sink);
      return;
    }
  }
  for (int k = 0; k < a.n_views; ++k) try_view<T, TRACE>(a, st, k, px, py, pz, dx, dy, dz, v, sink);
}

template <typename T, bool TRACE>
__global__ void __launch_bounds__(256) transport_kernel(const TArgs<T> a) {
  __shared__ T s_c0[256], s_c1[256], s_c2[256];
  __shared__ unsigned long long s_fates[4];
  for (int m = threadIdx.x; m < a.n_mat; m += blockDim.x) {
    s_c0[m] = a.coef[3 * m];
    s_c1[m] = a.coef[3 * m + 1];
    s_c2[m] = a.coef[3 * m + 2];
  }
  if (threadIdx.x < 4) s_fates[threadIdx.x] = 0ull;
  __syncthreads();

  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint32_t stride_mod = (uint32_t)(stride % a.n_vox);
  uint64_t i = tid;
  uint32_t v = (uint32_t)((a.first + tid) % a.n_vox);  // voxel of history first + i
  const uint32_t nxy = (uint32_t)a.nx * (uint32_t)a.ny;

  Stream st;
  T px = 0, py = 0, pz = 0, dx = 0, dy = 0, dz = 1;
  Energy<T> en;
  en.e = en.sig = en.e3 = en.ie3 = (T)0;
  uint32_t steps = 0, n_virtual = 0, n_real = 0, n_compton = 0;
  uint32_t cur_v = 0;
  uint64_t cur_i = 0;
  bool alive = false;
  mc_history_record rec;
  EventSink sink{a.events, a.cursor, a.capacity, &rec};

  for (;;) {
    int fate = -1;
    if (!alive) {
      if (i >= a.count) break;
      // emission (Sec. 3, isotropic 4 pi): uniform point in voxel v, uniform direction
      cur_i = i;
      cur_v = v;
      st.init(a.key0, a.key1, a.first + i);
      i += stride;
      v += stride_mod;
      if (v >= a.n_vox) v -= a.n_vox;
      const uint32_t vi = cur_v % (uint32_t)a.nx;
      const uint32_t vj = (cur_v / (uint32_t)a.nx) % (uint32_t)a.ny;
      const uint32_t vk = cur_v / nxy;
      px = ((T)vi + uniform<T>(st.word())) * a.h - a.hx;
      py = ((T)vj + uniform<T>(st.word())) * a.h - a.hy;
      pz = ((T)vk + uniform<T>(st.word())) * a.h - a.hz;
      const T ct = (T)2 * uniform<T>(st.word()) - (T)1;
      T cph, sph;
      cos_sin_2pi<T>(uniform<T>(st.word()), cph, sph);
      const T sth = sqrt(fmax((T)0, (T)1 - ct * ct));
      dx = sth * cph;
      dy = sth * sph;
      dz = ct;
      en.set(a.e0);
      steps = n_virtual = n_real = n_compton = 0;
      alive = true;
      if (TRACE) {
        rec.n_events = 0;
      }
      if (!(a.mu_maj > (T)0)) fate = MC_FATE_ESCAPE;
    }
    if (fate < 0) {
      // one Woodcock flight over the majorant
      if (steps >= kStepCap) {
        fate = MC_FATE_CAP;
      } else {
        steps += 1;
        const T s = neg_log<T>(uniform<T>(st.word())) / a.mu_maj;
        const T qx = px + s * dx, qy = py + s * dy, qz = pz + s * dz;
        if (!(qx >= -a.hx && qx < a.hx && qy >= -a.hy && qy < a.hy && qz >= -a.hz && qz < a.hz)) {
          fate = MC_FATE_ESCAPE;  // leaves from the pre-flight point p
        } else {
          px = qx; py = qy; pz = qz;
          const int ix = (int)voxel_index<T>(px, a.hx, a.h, a.nx);
          const int iy = (int)voxel_index<T>(py, a.hy, a.h, a.ny);
          const int iz = (int)voxel_index<T>(pz, a.hz, a.h, a.nz);
          const int m = __ldg(a.mat + ((size_t)iz * a.ny + iy) * a.nx + ix);
          const T mu = mu_total<T>(s_c0, s_c1, s_c2, m, en);
          if (uniform<T>(st.word()) * a.mu_maj < mu) {
            n_real += 1;
            if (uniform<T>(st.word()) * mu < mu_photo<T>(s_c0, s_c1, s_c2, m, en)) {
              fate = MC_FATE_ABSORBED;
            } else {
              T mu_c, eps;
              if (!compton<T>(st, en.e, mu_c, eps)) {
                fate = MC_FATE_CAP;
              } else {
                T cp, sp;
                cos_sin_2pi<T>(uniform<T>(st.word()), cp, sp);
                rotate<T>(dx, dy, dz, mu_c, cp, sp);
                const T e_new = eps * en.e;
                n_compton += 1;
                if (e_new < a.e_low) {
                  en.e = e_new;
                  fate = MC_FATE_BELOW_WINDOW;
                } else {
                  en.set(e_new);
                }
              }
            }
          } else {
            n_virtual += 1;
          }
        }
      }
    }
    if (fate >= 0) {
      if (fate == MC_FATE_ESCAPE) detect<T, TRACE>(a, st, px, py, pz, dx, dy, dz, cur_v, sink);
      atomicAdd(&s_fates[fate], 1ull);
      if (TRACE) {
        rec.fate = (uint8_t)fate;
        rec.pad = 0;
        rec.n_virtual = n_virtual;
        rec.n_real = n_real;
        rec.n_compton = n_compton;
        rec.n_draws = st.n_draws;
        rec.pad2 = 0;
        rec.e_final_kev = (double)en.e;
        for (int e = rec.n_events; e < 4; ++e) rec.event_row[e] = 0;
        a.records[cur_i] = rec;
      }
      alive = false;
    }
  }
  __syncthreads();
  if (threadIdx.x < 4 && s_fates[threadIdx.x]) atomicAdd(&a.fates[threadIdx.x], s_fates[threadIdx.x]);
}

// Compton sampler alone (verification).
template <typename T>
__global__ void debug_kn_kernel(T e, uint32_t k0, uint32_t k1, uint64_t n, double *cos_out, double *eps_out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    Stream st;
    st.init(k0, k1, i);
    T mu = 0, eps = 0;
    compton<T>(st, e, mu, eps);
    cos_out[i] = (double)mu;
    eps_out[i] = (double)eps;
  }
}

// Woodcock flight alone (verification): photons from p0 along d, counts
// those that leave the grid without a real collision.
template <typename T>
__global__ void debug_beam_kernel(const TArgs<T> a, T p0x, T p0y, T p0z, T dx, T dy, T dz, T e, uint64_t n,
                                  unsigned long long *through) {
  __shared__ T s_c0[256], s_c1[256], s_c2[256];
  for (int m = threadIdx.x; m < a.n_mat; m += blockDim.x) {
    s_c0[m] = a.coef[3 * m];
    s_c1[m] = a.coef[3 * m + 1];
    s_c2[m] = a.coef[3 * m + 2];
  }
  __syncthreads();
  Energy<T> en;
  en.set(e);
  unsigned long long mine = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!(a.mu_maj > (T)0)) { mine += 1; continue; }
    Stream st;
    st.init(a.key0, a.key1, i);
    T px = p0x, py = p0y, pz = p0z;
    for (uint32_t s = 0; s < kStepCap; ++s) {
      const T l = neg_log<T>(uniform<T>(st.word())) / a.mu_maj;
      const T qx = px + l * dx, qy = py + l * dy, qz = pz + l * dz;
      if (!(qx >= -a.hx && qx < a.hx && qy >= -a.hy && qy < a.hy && qz >= -a.hz && qz < a.hz)) { mine += 1; break; }
      px = qx; py = qy; pz = qz;
      const int ix = (int)voxel_index<T>(px, a.hx, a.h, a.nx);
      const int iy = (int)voxel_index<T>(py, a.hy, a.h, a.ny);
      const int iz = (int)voxel_index<T>(pz, a.hz, a.h, a.nz);
      const int m = a.mat[((size_t)iz * a.ny + iy) * a.nx + ix];
      if (uniform<T>(st.word()) * a.mu_maj < mu_total<T>(s_c0, s_c1, s_c2, m, en)) break;
    }
  }
  if (mine) atomicAdd(through, mine);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
constexpr double kAvogadro = 6.02214076e23;

// Host copy of the attenuation model, evaluated in the same order as on the
// device in double mode: 0.1 rho (N_A (Z/A) sigma_KN(E) + k Z^4 / E^3).
inline double host_sigma_kn(double e) {
  const double a = e / kMec2;
  const double t = 1.0 + 2.0 * a;
  const double l = std::log(t);
  const double term1 = (1.0 + a) / (a * a) * (2.0 * (1.0 + a) / t - l / a);
  const double term2 = l / (2.0 * a);
  const double term3 = (1.0 + 3.0 * a) / (t * t);
  return 2.0 * kPi * kRe * kRe * (term1 + term2 - term3);
}

inline double host_mu(const TransportSetup &ts, int m, double e) {
  const double z = ts.zeff[m];
  const double z4 = (z * z) * (z * z);
  const double compton = kAvogadro * ts.zoa[m] * host_sigma_kn(e);
  const double photo = ts.photo_k * z4 / (e * e * e);
  return 0.1 * ts.rho[m] * (compton + photo);
}

inline double host_e_low(const TransportSetup &ts) { return (1.0 - 0.5 * ts.window) * ts.e0; }

inline double host_majorant(const TransportSetup &ts) {
  const double el = host_e_low(ts);
  double best = 0.0;
  for (int m = 0; m < ts.n_mat; ++m) {
    const double mu = host_mu(ts, m, el);
    if (mu > best) best = mu;
  }
  return best;
}

// Per-material coefficients of the attenuation model for each precision:
// double {0.1 rho, N_A Z/A, k Z^4} (evaluated as written on the device),
// float {0.1 rho N_A Z/A, 0.1 rho k Z^4, 0}.
inline void host_coefficients(const TransportSetup &ts, std::vector<double> &cd, std::vector<float> &cf) {
  cd.assign(3 * (size_t)ts.n_mat, 0.0);
  cf.assign(3 * (size_t)ts.n_mat, 0.0f);
  for (int m = 0; m < ts.n_mat; ++m) {
    const double r01 = 0.1 * ts.rho[m];
    const double nazoa = kAvogadro * ts.zoa[m];
    const double z = ts.zeff[m];
    const double kz4 = ts.photo_k * ((z * z) * (z * z));
    cd[3 * m] = r01; cd[3 * m + 1] = nazoa; cd[3 * m + 2] = kz4;
    cf[3 * m] = (float)(r01 * nazoa); cf[3 * m + 1] = (float)(r01 * kz4); cf[3 * m + 2] = 0.0f;
  }
}

template <typename T> void make_targs(const TransportSetup &ts, TArgs<T> &a) {
  a.coef = std::is_same<T, double>::value ? (const T *)(const void *)ts.coef_d_dev
                                          : (const T *)(const void *)ts.coef_f_dev;
  a.mat = ts.material_dev;
  a.view_cs = std::is_same<T, double>::value ? (const T *)(const void *)ts.view_cs_dev
                                             : (const T *)(const void *)ts.view_cs_f_dev;
  a.nx = ts.nx; a.ny = ts.ny; a.nz = ts.nz; a.n_mat = ts.n_mat;
  a.h = (T)ts.h;
  a.hx = (T)(0.5 * ts.nx * ts.h);
  a.hy = (T)(0.5 * ts.ny * ts.h);
  a.hz = (T)(0.5 * ts.nz * ts.h);
  a.mu_maj = (T)host_majorant(ts);
  a.e0 = (T)ts.e0;
  a.e_low = (T)host_e_low(ts);
  const double ratio = ts.hole_len / ts.hole_diam;
  a.ratio = (T)ratio;
  const double tan_max = ts.hole_diam / ts.hole_len;
  a.w_max = (T)(tan_max / std::sqrt(1.0 + tan_max * tan_max) * 1.02 + 1e-6);
  const double delta = ts.arc_deg / ts.n_views;
  a.start_deg = (T)ts.start_deg;
  a.inv_delta = (T)(1.0 / delta);
  a.psi_views = (T)(std::atan(tan_max) * (180.0 / kPi) * 1.02 / std::fabs(delta) + 1e-6);
  a.views_per_turn = 0;
  if (delta > 0.0 && ts.arc_deg <= 360.0) {
    const double kt = 360.0 / delta;
    const double kr = std::floor(kt + 0.5);
    if (std::fabs(kt - kr) < 1e-9 * kt && kr >= ts.n_views && kr < 2147483647.0) a.views_per_turn = (int)kr;
  }
  a.sigma = (T)(ts.fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0))));
  a.plane = (T)(ts.radius_mm + ts.hole_len);
  a.bin = (T)ts.bin_mm;
  a.half_bu = (T)(0.5 * ts.bins_u);
  a.half_bv = (T)(0.5 * ts.bins_v);
  a.n_views = ts.n_views; a.bins_u = ts.bins_u; a.bins_v = ts.bins_v;
  a.n_vox = (uint32_t)((uint64_t)ts.nx * ts.ny * ts.nz);
  a.n_rows = (uint64_t)ts.n_views * ts.bins_u * ts.bins_v;
  a.first = ts.first; a.count = ts.count;
  a.key0 = ts.key0; a.key1 = ts.key1;
  a.events = ts.events; a.capacity = ts.capacity; a.cursor = ts.cursor; a.fates = ts.fates;
  a.records = ts.records;
}

template <typename T> int launch_transport_t(const TransportSetup &ts, cudaStream_t s) {
  TArgs<T> a;
  make_targs<T>(ts, a);
  if (ts.count == 0) return MC_OK;
  const int threads = 256;
  int per_sm = 0;
  if (ts.records) {
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_kernel<T, true>, threads, 0));
  } else {
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_kernel<T, false>, threads, 0));
  }
  if (per_sm < 1) per_sm = 1;
  const int64_t full = (int64_t)device_sm_count() * per_sm;
  const int64_t need = (int64_t)((ts.count + threads - 1) / threads);
  const int grid = (int)(need < full ? need : full);
  if (ts.records) { count_launch(); transport_kernel<T, true><<<grid, threads, 0, s>>>(a); }
  else { count_launch(); transport_kernel<T, false><<<grid, threads, 0, s>>>(a); }
  MCS_LAUNCHED();
  return MC_OK;
}

template <typename T>
int launch_debug_kn_t(double e_kev, uint64_t seed, uint64_t n, double *cos_dev, double *eps_dev, cudaStream_t s) {
  if (n == 0) return MC_OK;
  const int threads = 256;
  const int64_t need = (int64_t)((n + threads - 1) / threads);
  const int grid = (int)(need < 4096 ? need : 4096);
  count_launch(); debug_kn_kernel<T><<<grid, threads, 0, s>>>((T)e_kev, (uint32_t)seed, (uint32_t)(seed >> 32), n, cos_dev, eps_dev);
  MCS_LAUNCHED();
  return MC_OK;
}

template <typename T>
int launch_debug_beam_t(const TransportSetup &ts, uint64_t n, const double p0[3], const double d[3], double e_kev,
                        unsigned long long *through_dev, cudaStream_t s) {
  TArgs<T> a;
  make_targs<T>(ts, a);
  if (n == 0) return MC_OK;
  const int threads = 256;
  const int64_t need = (int64_t)((n + threads - 1) / threads);
  const int grid = (int)(need < 4096 ? need : 4096);
  count_launch(); debug_beam_kernel<T><<<grid, threads, 0, s>>>(a, (T)p0[0], (T)p0[1], (T)p0[2], (T)d[0], (T)d[1], (T)d[2],
                                                (T)e_kev, n, through_dev);
  MCS_LAUNCHED();
  MCS_CUDA(cudaStreamSynchronize(s));
  return MC_OK;
}

}  // namespace mcs
