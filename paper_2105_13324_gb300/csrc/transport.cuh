// transport.cuh -- persistent photon-history kernel (paper Sec. 2: follow
// each source photon until it is absorbed, leaves the energy window or
// escapes, sampling every step from the cross-sections; Sec. 3: parallel-hole
// collimation and the detection window; Sec. 5.1: the detections estimate the
// response matrix T_ij of Eq. (IMC)).
//
// Included by transport_f32.cu (production, float) and transport_f64.cu
// (verification, double, compiled with --fmad=false so that every product and
// sum is rounded as written and the per-history trace can be compared with a
// double-precision reference).  The double path evaluates every formula of the
// transport contract literally (divisions, the closed-form cross-section);
// the float path computes the same quantities with cheaper operations
// (reciprocal multiplies, rsqrt, a cross-section table over the energy
// window) -- the draws consumed and the decisions taken are the same, up to
// rounding.
//
// One thread follows one history at a time; when its history ends it starts
// the next one of its grid-stride sequence (lane refill), so the warps stay
// full until the last histories of the launch.  Each loop iteration is up to
// two Woodcock flights (the second after a virtual collision).
#pragma once

#include <cooperative_groups.h>

#include <cmath>
#include <cstring>
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
constexpr int kSigTab = 256;              // float path: sigma_KN table over [E_low, E0]
constexpr int kWaitCollide = 12;          // lanes waiting at a real collision before a warp handles them
constexpr int kWaitEmit = 8;             // lanes waiting for a new history before a warp emits

template <typename T> struct TArgs {
  const uint8_t *mat;
  const T *coef;     // per material: double {0.1 rho, N_A Z/A, k Z^4}; float {0.1 rho N_A Z/A, 0.1 rho k Z^4}
  const T *view_cs;  // [2V] cos, sin of theta_k
  const float *sig_tab;  // [kSigTab] sigma_KN at E_low + i (E0 - E_low)/(kSigTab - 1)
  const uint8_t *skip;   // float forced detection: distance map of the material grid
  uint32_t rk[20];   // Philox round keys: round r uses (rk[2r], rk[2r+1])
  int nx, ny, nz, n_mat;
  T h, hx, hy, hz;   // voxel size, half extents
  T inv_h, hx_h, hy_h, hz_h;  // 1/h and the half extents in voxels (float path)
  T mu_maj, inv_mu_maj, e0, e_low, inv_de;
  T ratio;           // L / d
  T w_max;           // |d_z| bound above which no view can accept (with margin)
  T start_deg, inv_delta, psi_views;  // azimuth window of candidate views
  int views_per_turn;                 // 360 / delta if integral, else 0
  int t_coll, t_emit;                 // lanes that must wait before a warp runs collisions / emissions
  uint64_t stride;                    // threads in the grid
  uint32_t step_v[3];                 // stride mod N as a voxel step (x, y, z)
  int primary_only;                   // tally only photons that never scattered
  T sigma, plane, bin, half_bu, half_bv;
  int n_views, bins_u, bins_v;
  uint32_t n_vox;
  uint64_t n_rows;
  uint64_t first, count;
  unsigned long long *events;
  unsigned long long capacity;
  unsigned long long *cursor;
  unsigned long long *fates;
  mc_history_record *records;
  void *esc;                        // EscapeRec<T>[esc_capacity] (forced detection: FdRec<T>)
  unsigned long long esc_capacity;
  unsigned long long *esc_cursor;
  unsigned long long *weights;      // forced detection: fixed-point event weights
  T cos_max, omega, omega_4pi;      // acceptance cone: cos of its half-angle, solid angle, / 4 pi
  T one_m_cos_max;                  // 1 - cos_max (float path: sin^2 from 1 - cos without cancellation)
  int forced_dir;                   // forced emission direction: cos(theta) in (-band, band)
  T band;                           // sin of the acceptance half-angle
  unsigned long long q_dir;         // fixed-point weight of a detection under forced direction
};

// An escaping photon that may pass a collimator: its history, the position
// of its random stream (words drawn so far) and its exit point and direction.
template <typename T> struct EscapeRec {
  uint64_t h;
  uint32_t n_draws, pad;  // words of the history's stream used so far
  T p[3], d[3];
};
static_assert(sizeof(EscapeRec<float>) == 40 && sizeof(EscapeRec<double>) == 64, "escape record layout");

// Forced detection: one interaction location of a history -- its emission
// (n = 0) or its n-th real collision -- with the photon's energy and
// direction before the interaction and the probability 1 - mu_pe/mu that
// the photon is not absorbed there (1 at emission).
template <typename T> struct FdRec {
  uint64_t h;
  uint32_t n, pad;
  T p[3], d[3];
  T e, keep;
};
static_assert(sizeof(FdRec<float>) == 48 && sizeof(FdRec<double>) == 80, "forced-detection record layout");

// Philox4x32-10 with precomputed round keys (Salmon et al., SC'11): each
// round is two 32x32->64 multiplies and two three-way xors.  The R-argument
// form runs rounds R..9 only, for a caller that has done rounds 0..R-1.
template <int R>
__device__ __forceinline__ void philox_rounds_from(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                                   const uint32_t *rk) {
#pragma unroll
  for (int r = R; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk[2 * r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk[2 * r + 1];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
}
__device__ __forceinline__ void philox_rounds(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3,
                                              const uint32_t *rk) {
  philox_rounds_from<0>(c0, c1, c2, c3, rk);
}

// One history's stream: block b of history h is counter (b, 0, h_lo, h_hi);
// words are consumed w0, w1, w2, w3, then the next block.
struct KStream {
  uint32_t h_lo, h_hi, block, w0, w1, w2, w3, left, n_draws;
  __device__ __forceinline__ void init(uint64_t h) {
    h_lo = (uint32_t)h; h_hi = (uint32_t)(h >> 32);
    block = 0; left = 0; n_draws = 0;
  }
  __device__ __forceinline__ uint32_t word(const uint32_t *rk) {
    if (left == 0) {
      uint32_t c0 = block, c1 = 0u, c2 = h_lo, c3 = h_hi;
      philox_rounds(c0, c1, c2, c3, rk);
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

// KStream with its round keys, as a draw source.
struct KRng {
  KStream &s;
  const uint32_t *rk;
  __device__ __forceinline__ void need(uint32_t) {}
  __device__ __forceinline__ uint32_t next() { return s.word(rk); }
};

// Per-thread ring of 16 stream words in shared memory, laid out slot-major
// (ring[slot][thread]) so that a warp's accesses never conflict whatever slot
// each lane is at.  ensure(k) tops the ring up (one Philox block) when fewer
// than k words are left, and is called before each group of draws, so blocks
// are generated where most lanes need them and no word is generated past
// the end of a history.  The stream position is 4 * blocks - words left.
// The head starts at slot 0 with each history, so block b always lands in
// slots 4 (b mod 4) .. 4 (b mod 4) + 3 (head + words left = 4 b mod 16).
constexpr int kRing = 16;
constexpr int kRingThreads = 256;
template <typename T> struct TArgs;

// Ring's Philox: block b's counter is (b, 0, h_lo, h_hi).  Round 0 turns it into
// (u0, u1, hi(M0 b) ^ h_hi ^ k1_0, lo(M0 b)) with u0 = hi(M1 h_lo) ^ k0_0 and
// u1 = lo(M1 h_lo), which depend on the history only; round 1 then forms
// M0 u0, again the history's alone.  start() computes those once per history
// (hk, e1 = u1 ^ k0_1, f1 = hi(M0 u0) ^ k1_1, d1 = lo(M0 u0)), so a refill
// does two multiplies for rounds 0 and 1 instead of four; the words are the
// same as from philox_rounds on the full counter.
struct Ring {
  uint32_t (*buf)[kRingThreads];
  uint32_t tid, head, avail, blk;
  uint32_t hk, e1, f1, d1;
  __device__ __forceinline__ void start(uint64_t h, const uint32_t *rk) {
    const uint32_t h_lo = (uint32_t)h, h_hi = (uint32_t)(h >> 32);
    blk = 0; avail = 0; head = 0;
    const uint64_t m1 = (uint64_t)0xCD9E8D57u * h_lo;
    const uint64_t m0 = (uint64_t)0xD2511F53u * ((uint32_t)(m1 >> 32) ^ rk[0]);
    hk = h_hi ^ rk[1];
    e1 = (uint32_t)m1 ^ rk[2];
    f1 = (uint32_t)(m0 >> 32) ^ rk[3];
    d1 = (uint32_t)m0;
  }
  template <typename A> __device__ __forceinline__ void refill(const A &a) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * blk;         // round 0's block-dependent half
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * ((uint32_t)(p0 >> 32) ^ hk);  // round 1
    uint32_t c0 = (uint32_t)(p1 >> 32) ^ e1, c1 = (uint32_t)p1, c2 = f1 ^ (uint32_t)p0, c3 = d1;
    philox_rounds_from<2>(c0, c1, c2, c3, a.rk);
    uint32_t *w = &buf[(blk & 3u) << 2][tid];  // four rows from here
    w[0] = c0;
    w[kRingThreads] = c1;
    w[2 * kRingThreads] = c2;
    w[3 * kRingThreads] = c3;
    avail += 4;
    blk += 1;
  }
  template <typename A> __device__ __forceinline__ void ensure(uint32_t k, const A &a) {
    if (avail < k) refill(a);
  }
  __device__ __forceinline__ uint32_t next() {
    const uint32_t w = buf[head][tid];
    head = (head + 1) & (kRing - 1);
    avail -= 1;
    return w;
  }
  __device__ __forceinline__ uint32_t n_draws() const { return 4u * blk - avail; }
};

// Ring bound to the launch's round keys, as a draw source for the samplers.
template <typename A> struct RingRng {
  Ring &r;
  const A &a;
  __device__ __forceinline__ void need(uint32_t k) { r.ensure(k, a); }
  __device__ __forceinline__ uint32_t next() { return r.next(); }
};

template <typename T> constexpr bool is_dbl() { return std::is_same<T, double>::value; }

// Klein-Nishina total cross-section per electron, cm^2, in the order
// 2 pi re re ((1+a)/(a a) (2(1+a)/t - l/a) + l/(2a) - (1+3a)/(t t)),
// a = E/mc^2, t = 1 + 2a, l = ln t.
__device__ __forceinline__ double sigma_kn(double e) {
  const double a = e / kMec2;
  const double t = 1.0 + 2.0 * a;
  const double l = log(t);
  const double term1 = (1.0 + a) / (a * a) * (2.0 * (1.0 + a) / t - l / a);
  const double term2 = l / (2.0 * a);
  const double term3 = (1.0 + 3.0 * a) / (t * t);
  return (2.0 * kPi) * kRe * kRe * (term1 + term2 - term3);
}

// Photon energy with the cross-section quantities that depend on it.
template <typename T> struct Energy {
  T e, sig, e3, ie3;
  __device__ __forceinline__ void set(T v, const TArgs<T> &a, const float *tab) {
    e = v;
    if constexpr (is_dbl<T>()) {
      sig = sigma_kn(v);
      e3 = v * v * v;
    } else {
      float t = (v - a.e_low) * a.inv_de;
      t = fminf(fmaxf(t, 0.0f), (float)(kSigTab - 1));
      const int i = min((int)t, kSigTab - 2);
      const float f = t - (float)i;
      sig = fmaf(f, tab[i + 1] - tab[i], tab[i]);
      const float ie = __fdividef(1.0f, v);
      ie3 = ie * ie * ie;
    }
  }
};

// mu(m, E) and mu_photo(m, E) in 1/mm.
template <typename T>
__device__ __forceinline__ T mu_total(const T *c0, const T *c1, const T *c2, int m, const Energy<T> &en) {
  if constexpr (is_dbl<T>()) return c0[m] * (c1[m] * en.sig + c2[m] / en.e3);
  else return fmaf(c0[m], en.sig, c1[m] * en.ie3);
}
template <typename T>
__device__ __forceinline__ T mu_photo(const T *c0, const T *c1, const T *c2, int m, const Energy<T> &en) {
  if constexpr (is_dbl<T>()) return c0[m] * (c2[m] / en.e3);
  else return c1[m] * en.ie3;
}

// Flight length -ln(u) / mu_maj.
template <typename T> __device__ __forceinline__ T flight(T u, const TArgs<T> &a) {
  if constexpr (is_dbl<T>()) return -log(u) / a.mu_maj;
  else return -__logf(u) * a.inv_mu_maj;
}

// cos and sin of phi = 2 pi u.
template <typename T> __device__ __forceinline__ void cos_sin_2pi(T u, T &c, T &s) {
  if constexpr (is_dbl<T>()) {
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

// sqrt(max(0, x))
template <typename T> __device__ __forceinline__ T sqrt0(T x) {
  if constexpr (is_dbl<T>()) return sqrt(fmax(0.0, x));
  else return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

// Voxel index along one axis: min(floor((x + half) / h), n - 1), x >= -half.
template <typename T> __device__ __forceinline__ int voxel_index(T x, T half, T h, T inv_h, T half_h, int n) {
  if constexpr (is_dbl<T>()) {
    const double f = floor((x + half) / h);
    return (int)(f > (double)(n - 1) ? (double)(n - 1) : f);
  } else {
    const int i = __float2int_rd(fmaf(x, inv_h, half_h));
    return max(0, min(i, n - 1));
  }
}

// Compton scatter by rejection: mu uniform in [-1,1], eps = 1/(1 + a(1-mu)),
// accepted with probability eps^2 (eps + 1/eps - (1 - mu^2)) / 2 (the
// Klein-Nishina density over its maximum).
template <typename T, typename R>
__device__ __forceinline__ bool compton(R &rng, T e, T &mu_out, T &eps_out) {
  T alpha;
  if constexpr (is_dbl<T>()) alpha = e / kMec2;
  else alpha = e * (float)(1.0 / kMec2);
  for (uint32_t t = 0; t < kTrialCap; ++t) {
    rng.need(2);
    const T mu = (T)2 * uniform<T>(rng.next()) - (T)1;
    const T den = (T)1 + alpha * ((T)1 - mu);
    T eps, f;
    if constexpr (is_dbl<T>()) {
      eps = 1.0 / den;
      f = 0.5 * eps * eps * (eps + 1.0 / eps - (1.0 - mu * mu));
    } else {
      eps = __fdividef(1.0f, den);
      f = 0.5f * eps * eps * (eps + den - (1.0f - mu * mu));
    }
    if (uniform<T>(rng.next()) < f) {
      mu_out = mu;
      eps_out = eps;
      return true;
    }
  }
  return false;
}

// Turn direction d by polar cosine mu and azimuth phi about itself.
template <typename T> __device__ __forceinline__ void rotate(T &u, T &v, T &w, T mu, T cp, T sp) {
  if constexpr (is_dbl<T>()) {
    const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
    double nu, nv, nw;
    if (fabs(w) < 0.99999) {
      const double r = sqrt(1.0 - w * w);
      nu = mu * u + st * (u * w * cp - v * sp) / r;
      nv = mu * v + st * (v * w * cp + u * sp) / r;
      nw = mu * w - st * cp * r;
    } else {
      nu = st * cp;
      nv = st * sp;
      nw = (w >= 0.0 ? mu : -mu);
    }
    const double n = sqrt(nu * nu + nv * nv + nw * nw);
    u = nu / n;
    v = nv / n;
    w = nw / n;
  } else {
    const float st = sqrt0<float>(1.0f - mu * mu);
    float nu, nv, nw;
    if (fabsf(w) < 0.99999f) {
      const float r2 = 1.0f - w * w;
      const float ri = rsqrtf(r2);
      const float sr = st * ri;
      nu = fmaf(mu, u, sr * (u * w * cp - v * sp));
      nv = fmaf(mu, v, sr * (v * w * cp + u * sp));
      nw = fmaf(mu, w, -st * cp * (r2 * ri));
    } else {
      nu = st * cp;
      nv = st * sp;
      nw = (w >= 0.0f ? mu : -mu);
    }
    const float ni = rsqrtf(nu * nu + nv * nv + nw * nw);
    u = nu * ni;
    v = nv * ni;
    w = nw * ni;
  }
}

struct EventSink {
  unsigned long long *events, *cursor;
  unsigned long long capacity;
  mc_history_record *rec;  // trace mode: the history's record
  unsigned long long *weights;  // weighted tallies (forced direction): one weight per event
  unsigned long long q;         // ... the weight of every detection
};

__device__ __forceinline__ void push_event(const EventSink &s, unsigned long long key) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(s.cursor, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  const unsigned long long idx = base + g.thread_rank();
  if (idx < s.capacity) {
    s.events[idx] = key;
    if (s.weights) s.weights[idx] = s.q;
  }
}

// The acceptance-cone test of try_view alone: view k can accept a photon
// moving along d (no draw).
template <typename T>
__device__ __forceinline__ bool in_cone(const TArgs<T> &a, int k, T dx, T dy) {
  const T ck = a.view_cs[2 * k], sk = a.view_cs[2 * k + 1];
  const T c = dx * ck + dy * sk;
  if (!(c > (T)0)) return false;
  const T stt = sqrt0<T>((T)1 - c * c);
  return a.ratio * stt < c;
}

// Offer view k to an escaping photon at p (inside the grid) moving along d.
template <typename T, bool TRACE>
__device__ __forceinline__ void try_view(const TArgs<T> &a, KStream &st, int k, T px, T py, T pz, T dx, T dy,
                                         T dz, uint32_t v, const EventSink &sink) {
  const T ck = a.view_cs[2 * k], sk = a.view_cs[2 * k + 1];
  const T c = dx * ck + dy * sk;
  if (!(c > (T)0)) return;
  const T stt = sqrt0<T>((T)1 - c * c);
  if (!(a.ratio * stt < c)) return;
  const T x = a.ratio * stt / c;
  const T pass = (T)(2.0 / kPi) * (acos(x) - x * sqrt0<T>((T)1 - x * x));
  if (!(uniform<T>(st.word(a.rk)) < pass)) return;
  const T t = (a.plane - (px * ck + py * sk)) / c;
  const T qx = px + t * dx, qy = py + t * dy, qz = pz + t * dz;
  T au = -qx * sk + qy * ck;
  T bv = qz;
  const T u1 = uniform<T>(st.word(a.rk));
  const T u2 = uniform<T>(st.word(a.rk));
  T r;
  if constexpr (is_dbl<T>()) r = sqrt(-2.0 * log(u1));
  else r = sqrt0<float>(-2.0f * __logf(u1));
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
// loop, in the same order.  The window's views are cone-tested first and the
// candidates then offered in order: each lane has one or two candidates
// among ~5 window views, so the expensive part of try_view runs once per
// candidate place of the warp instead of once per window view, with more
// lanes taking part each time.
template <typename T, bool TRACE>
__device__ __forceinline__ void detect(const TArgs<T> &a, KStream &st, T px, T py, T pz, T dx, T dy, T dz,
                                       uint32_t v, const EventSink &sink) {
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
      const int hi = kmax < K - 1 ? kmax : K - 1;
      // 1. the window's candidate views -- the cone test alone, no draws --
      // in ascending order, 8 bits each
      uint64_t list = 0ull;
      int nc = 0;
      bool full = false;
      auto consider = [&](int k) {
        if (in_cone<T>(a, k, dx, dy)) {
          if (nc < 8 && k < 256) {
            list |= (uint64_t)k << (8 * nc);
            ++nc;
          } else {
            full = true;
          }
        }
      };
      if (kmax >= K)
        for (int k = 0; k <= kmax - K && k < a.n_views; ++k) consider(k);
      for (int k = kmin; k <= hi && k < a.n_views; ++k) consider(k);
      if (!full) {
        // 2. the candidates in order with their draws: a warp runs this
        // once per candidate place rather than once per window view
        for (int t = 0; t < nc; ++t)
          try_view<T, TRACE>(a, st, (int)((list >> (8 * t)) & 255u), px, py, pz, dx, dy, dz, v, sink);
        return;
      }
      if (kmax >= K) {
        for (int k = 0; k <= kmax - K && k < a.n_views; ++k) try_view<T, TRACE>(a, st, k, px, py, pz, dx, dy, dz, v, sink);
      }
      for (int k = kmin; k <= hi && k < a.n_views; ++k) try_view<T, TRACE>(a, st, k, px, py, pz, dx, dy, dz, v, sink);
      return;
    }
  }
  for (int k = 0; k < a.n_views; ++k) try_view<T, TRACE>(a, st, k, px, py, pz, dx, dy, dz, v, sink);
}

// Queue an interaction location for the forced-detection kernel.
template <typename T>
__device__ __forceinline__ void push_fd(const TArgs<T> &a, uint64_t h, uint32_t n, T px, T py, T pz, T dx, T dy,
                                        T dz, T e, T keep) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(a.esc_cursor, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  const unsigned long long q = base + g.thread_rank();
  if (q < a.esc_capacity) {
    FdRec<T> r;
    r.h = h; r.n = n; r.pad = 0;
    r.p[0] = px; r.p[1] = py; r.p[2] = pz;
    r.d[0] = dx; r.d[1] = dy; r.d[2] = dz;
    r.e = e; r.keep = keep;
    static_cast<FdRec<T> *>(a.esc)[q] = r;
  }
}

// FD: forced-detection mode -- instead of queueing escapes for analog
// detection, queue every interaction location (emission, real collisions).
template <typename T, bool TRACE, bool FD = false>
__global__ void __launch_bounds__(kRingThreads) transport_kernel(const __grid_constant__ TArgs<T> a) {
  __shared__ T s_c0[256], s_c1[256], s_c2[256];
  __shared__ float s_sig[kSigTab];
  __shared__ unsigned long long s_fates[4];
  __shared__ uint32_t s_ring[kRing][kRingThreads];
  for (int m = threadIdx.x; m < a.n_mat; m += blockDim.x) {
    s_c0[m] = a.coef[3 * m];
    s_c1[m] = a.coef[3 * m + 1];
    s_c2[m] = a.coef[3 * m + 2];
  }
  if (!is_dbl<T>())
    for (int i = threadIdx.x; i < kSigTab; i += blockDim.x) s_sig[i] = a.sig_tab[i];
  if (threadIdx.x < 4) s_fates[threadIdx.x] = 0ull;
  __syncthreads();
  // the emission energy's cross-section quantities, once per block
  __shared__ T s_en0[4];
  if (threadIdx.x == 0) {
    Energy<T> e0;
    e0.e = e0.sig = e0.e3 = e0.ie3 = (T)0;
    e0.set(a.e0, a, s_sig);
    s_en0[0] = e0.e; s_en0[1] = e0.sig; s_en0[2] = e0.e3; s_en0[3] = e0.ie3;
  }
  __syncthreads();

  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = a.stride;
  // voxel of the next history, kept as (vi, vj, vk) and advanced by the
  // stride (mod N) with carries
  const uint32_t nx = (uint32_t)a.nx, ny = (uint32_t)a.ny, nz = (uint32_t)a.nz;
  uint32_t vi, vj, vk;
  const uint32_t si = a.step_v[0], sj = a.step_v[1], sk = a.step_v[2];
  {
    const uint32_t v0 = (uint32_t)((a.first + tid) % a.n_vox);
    vi = v0 % nx; vj = (v0 / nx) % ny; vk = v0 / (nx * ny);
  }
  uint64_t i = tid;

  Ring rg;
  rg.buf = s_ring;
  rg.tid = threadIdx.x;
  rg.head = 0;
  rg.start(a.first + i, a.rk);
  T px = 0, py = 0, pz = 0, dx = 0, dy = 0, dz = 1;
  Energy<T> en;
  en.e = en.sig = en.e3 = en.ie3 = (T)0;
  uint32_t steps = 0, n_virtual = 0, n_real = 0, n_compton = 0;
  uint64_t cur_i = 0;
  uint32_t n_fate[4] = {0u, 0u, 0u, 0u};  // fates of this thread's histories

  RingRng<TArgs<T>> rng{rg, a};
  // Lane states.  A lane that reaches a real collision, or needs a new
  // history, waits until at least t_coll (t_emit) lanes of its warp wait for
  // the same step -- or no lane is left flying -- so that the long collision
  // and emission steps run with many lanes at once while the others keep
  // flying.  All 32 lanes run every iteration (warp-uniform loop).
  enum { S_FLY = 0, S_COLLIDE = 1, S_EMIT = 2, S_DONE = 3 };
  int st = (i < a.count) ? S_EMIT : S_DONE;
  int m_col = 0;      // material at the pending real collision
  T mu_col = (T)0;    // and its attenuation
  for (;;) {
    const unsigned m_emit = __ballot_sync(0xffffffffu, st == S_EMIT);
    const unsigned m_coll = __ballot_sync(0xffffffffu, st == S_COLLIDE);
    const unsigned m_fly = __ballot_sync(0xffffffffu, st == S_FLY);
    if ((m_emit | m_coll | m_fly) == 0u) break;
    const bool do_coll = m_coll != 0u && (__popc(m_coll) >= a.t_coll || m_fly == 0u);
    const bool do_emit = m_emit != 0u && (__popc(m_emit) >= a.t_emit || m_fly == 0u);
    {
      // the one Philox point: words for everything this lane does below
      // (emission 5 + flight 2; collision: photo 1 + four rejection trials
      // 8 + azimuth 1 + flight 2; two flights 4; the ring's 16 words hold
      // any top-up of a lane below 12); a scatter needing more trials, or a
      // second flight after an emission or a collision, draws the rest inline
      uint32_t need = 0u;
      if (st == S_FLY) need = 4u;
      else if (st == S_EMIT && do_emit) need = 7u;
      else if (st == S_COLLIDE && do_coll) need = 12u;
      while (rg.avail < need) rg.refill(a);
    }
    int fate = -1;
    if (do_coll && st == S_COLLIDE) {
      if (FD && !a.primary_only)
        push_fd<T>(a, a.first + cur_i, n_real, px, py, pz, dx, dy, dz, en.e,
                   (T)1 - mu_photo<T>(s_c0, s_c1, s_c2, m_col, en) / mu_col);
      // photo-absorption, else a Klein-Nishina scatter, at the pending collision
      rg.ensure(1, a);
      if (uniform<T>(rg.next()) * mu_col < mu_photo<T>(s_c0, s_c1, s_c2, m_col, en)) {
        fate = MC_FATE_ABSORBED;
      } else {
        T mu_c, eps;
        if (!compton<T>(rng, en.e, mu_c, eps)) {
          fate = MC_FATE_CAP;
        } else {
          rg.ensure(1, a);
          T cp, sp;
          cos_sin_2pi<T>(uniform<T>(rg.next()), cp, sp);
          rotate<T>(dx, dy, dz, mu_c, cp, sp);
          const T e_new = eps * en.e;
          n_compton += 1;
          if (e_new < a.e_low) {
            en.e = e_new;
            fate = MC_FATE_BELOW_WINDOW;
          } else {
            en.set(e_new, a, s_sig);
            st = S_FLY;
          }
        }
      }
    }
    if (do_emit && st == S_EMIT) {
      // emission (Sec. 3, isotropic 4 pi): uniform point in voxel v, uniform
      // direction; five draws
      cur_i = i;
      px = ((T)vi + uniform<T>(rg.next())) * a.h - a.hx;
      py = ((T)vj + uniform<T>(rg.next())) * a.h - a.hy;
      pz = ((T)vk + uniform<T>(rg.next())) * a.h - a.hz;
      i += stride;
      vi += si;
      if (vi >= nx) { vi -= nx; vj += 1; }
      vj += sj;
      if (vj >= ny) { vj -= ny; vk += 1; }
      vk += sk;
      if (vk >= nz) vk -= nz;
      T ct = (T)2 * uniform<T>(rg.next()) - (T)1;
      if (a.forced_dir) ct = ct * a.band;  // only the band a collimator can see
      T cph, sph;
      cos_sin_2pi<T>(uniform<T>(rg.next()), cph, sph);
      const T sth = sqrt0<T>((T)1 - ct * ct);
      dx = sth * cph;
      dy = sth * sph;
      dz = ct;
      en.e = s_en0[0]; en.sig = s_en0[1]; en.e3 = s_en0[2]; en.ie3 = s_en0[3];
      steps = n_virtual = n_real = n_compton = 0;
      st = S_FLY;
      if (FD) push_fd<T>(a, a.first + cur_i, 0u, px, py, pz, dx, dy, dz, en.e, (T)1);
      if (!(a.mu_maj > (T)0)) fate = MC_FATE_ESCAPE;
    }
    // up to two Woodcock flights over the majorant: a lane whose first
    // flight ends in a virtual collision flies again in the same iteration
#pragma unroll 1
    for (int fl = 0; fl < 2 && st == S_FLY && fate < 0; ++fl) {
      if (steps >= kStepCap) {
        fate = MC_FATE_CAP;
      } else {
        steps += 1;
        rg.ensure(2, a);
        const T s = flight<T>(uniform<T>(rg.next()), a);
        const T qx = px + s * dx, qy = py + s * dy, qz = pz + s * dz;
        // float path: the box test on the voxel indices themselves (one
        // floor per axis, three unsigned compares); it can differ from the
        // coordinate test only by rounding at the grid's faces
        int ix, iy, iz;
        bool inside;
        if constexpr (is_dbl<T>()) {
          inside = qx >= -a.hx && qx < a.hx && qy >= -a.hy && qy < a.hy && qz >= -a.hz && qz < a.hz;
          ix = voxel_index<T>(qx, a.hx, a.h, a.inv_h, a.hx_h, a.nx);
          iy = voxel_index<T>(qy, a.hy, a.h, a.inv_h, a.hy_h, a.ny);
          iz = voxel_index<T>(qz, a.hz, a.h, a.inv_h, a.hz_h, a.nz);
        } else {
          ix = __float2int_rd(fmaf(qx, a.inv_h, a.hx_h));
          iy = __float2int_rd(fmaf(qy, a.inv_h, a.hy_h));
          iz = __float2int_rd(fmaf(qz, a.inv_h, a.hz_h));
          inside = (unsigned)ix < (unsigned)a.nx && (unsigned)iy < (unsigned)a.ny && (unsigned)iz < (unsigned)a.nz;
        }
        if (!inside) {
          fate = MC_FATE_ESCAPE;  // leaves from the pre-flight point p
        } else {
          px = qx; py = qy; pz = qz;
          // 32-bit index: grids hold fewer than 2^31 voxels
          const int m = __ldg(a.mat + (uint32_t)((iz * a.ny + iy) * a.nx + ix));
          const T mu = mu_total<T>(s_c0, s_c1, s_c2, m, en);
          if (uniform<T>(rg.next()) * a.mu_maj < mu) {
            n_real += 1;
            m_col = m;
            mu_col = mu;
            st = S_COLLIDE;
          } else {
            n_virtual += 1;
          }
        }
      }
    }
    if (fate >= 0) {
      if (!FD && fate == MC_FATE_ESCAPE && fabs(dz) < a.w_max && !(a.primary_only && n_compton > 0)) {
        // a view may accept it: queue it for the detection kernel
        cg::coalesced_group g = cg::coalesced_threads();
        unsigned long long base = 0;
        if (g.thread_rank() == 0) base = atomicAdd(a.esc_cursor, (unsigned long long)g.size());
        base = g.shfl(base, 0);
        const unsigned long long q = base + g.thread_rank();
        if (q < a.esc_capacity) {
          EscapeRec<T> e;
          e.h = a.first + cur_i;
          e.n_draws = rg.n_draws();
          e.pad = 0;
          e.p[0] = px; e.p[1] = py; e.p[2] = pz;
          e.d[0] = dx; e.d[1] = dy; e.d[2] = dz;
          static_cast<EscapeRec<T> *>(a.esc)[q] = e;
        }
      }
      n_fate[0] += fate == 0;
      n_fate[1] += fate == 1;
      n_fate[2] += fate == 2;
      n_fate[3] += fate == 3;
      if (TRACE) {
        mc_history_record rec;
        rec.fate = (uint8_t)fate;
        rec.n_events = 0;
        rec.pad = 0;
        rec.n_virtual = n_virtual;
        rec.n_real = n_real;
        rec.n_compton = n_compton;
        rec.n_draws = rg.n_draws();
        rec.pad2 = 0;
        rec.e_final_kev = (double)en.e;
        for (int e = 0; e < 4; ++e) rec.event_row[e] = 0;
        a.records[cur_i] = rec;
      }
      if (i < a.count) {
        st = S_EMIT;
        rg.start(a.first + i, a.rk);  // next history's stream
      } else {
        st = S_DONE;
      }
    }
  }
  // fates: warp sums, then one shared atomic per warp and fate
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    unsigned long long c = n_fate[f];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_fates[f], c);
  }
  __syncthreads();
  if (threadIdx.x < 4 && s_fates[threadIdx.x]) atomicAdd(&a.fates[threadIdx.x], s_fates[threadIdx.x]);
}

// Detection of the queued escapes (Sec. 3): each thread resumes one
// photon's random stream where transport left it and offers the photon to the
// views.  Trace mode adds the detections and draws to the history's record.
template <typename T, bool TRACE>
__global__ void __launch_bounds__(256) detect_kernel(const __grid_constant__ TArgs<T> a) {
  const unsigned long long n_q = *a.esc_cursor < a.esc_capacity ? *a.esc_cursor : a.esc_capacity;
  const EscapeRec<T> *q = static_cast<const EscapeRec<T> *>(a.esc);
  for (unsigned long long e = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_q;
       e += (unsigned long long)gridDim.x * blockDim.x) {
    const EscapeRec<T> r = q[e];
    KStream st;
    st.init(r.h);
    const uint32_t b = r.n_draws >> 2, used = r.n_draws & 3u;
    st.block = b;
    st.left = 0;
    if (used > 0) {
      uint32_t c0 = b, c1 = 0u, c2 = st.h_lo, c3 = st.h_hi;
      philox_rounds(c0, c1, c2, c3, a.rk);
      // the block's words not drawn yet
      if (used == 1) { st.w0 = c1; st.w1 = c2; st.w2 = c3; }
      else if (used == 2) { st.w0 = c2; st.w1 = c3; }
      else { st.w0 = c3; }
      st.left = 4 - used;
      st.block = b + 1;
    }
    st.n_draws = r.n_draws;
    const uint32_t v = (uint32_t)(r.h % a.n_vox);
    mc_history_record *rec = TRACE ? a.records + (r.h - a.first) : nullptr;
    EventSink sink{a.events, a.cursor, a.capacity, rec, a.forced_dir ? a.weights : nullptr, a.q_dir};
    detect<T, TRACE>(a, st, r.p[0], r.p[1], r.p[2], r.d[0], r.d[1], r.d[2], v, sink);
    if (TRACE) rec->n_draws = st.n_draws;
  }
}

// ---------------------------------------------------------------------------
// forced detection
// ---------------------------------------------------------------------------
// Transmission exp(-integral of mu(E) ds) from p along d to the grid
// boundary: the voxels the ray crosses are visited in order (the next voxel
// lies across the nearest of the three next faces, ties to the lowest axis)
// and mu times the length inside each is summed.
template <typename T>
__device__ __forceinline__ T transmission(const TArgs<T> &a, T px, T py, T pz, T dx, T dy, T dz, T e,
                                          const T *c0, const T *c1, const T *c2, const float *sig_tab) {
  Energy<T> en;
  en.set(e, a, sig_tab);
  if constexpr (!is_dbl<T>()) {
    // float path: the same integral, crossing a whole cube of constant mu per
    // step.  The distance map gives, for the current voxel, the half-width
    // D - 1 of the cube around it that holds one material; the ray leaves that
    // cube at the (D - 1)-th face beyond the voxel's own next face on one
    // axis, so mu times the length up to there is the exact integral over
    // the cube (D = 1 is one ordinary voxel step).  Face distances advance by
    // a constant step per axis, reciprocal multiplies replace divisions, and
    // the step has no branches.
    int ix = voxel_index<float>(px, a.hx, a.h, a.inv_h, a.hx_h, a.nx);
    int iy = voxel_index<float>(py, a.hy, a.h, a.inv_h, a.hy_h, a.ny);
    int iz = voxel_index<float>(pz, a.hz, a.h, a.inv_h, a.hz_h, a.nz);
    const int sx = dx > 0.0f ? 1 : (dx < 0.0f ? -1 : 0);
    const int sy = dy > 0.0f ? 1 : (dy < 0.0f ? -1 : 0);
    const int sz = dz > 0.0f ? 1 : (dz < 0.0f ? -1 : 0);
    const float rx = sx ? 1.0f / dx : 0.0f, ry = sy ? 1.0f / dy : 0.0f, rz = sz ? 1.0f / dz : 0.0f;
    // the first face on an axis lies at (i + (s > 0)) h - half, t = (face - p) / d;
    // each later face of that axis is h / |d| further along the ray
    const float ox = -a.hx - px, oy = -a.hy - py, oz = -a.hz - pz;
    float tx = sx ? fmaf((float)(ix + (sx > 0)), a.h, ox) * rx : INFINITY;
    float ty = sy ? fmaf((float)(iy + (sy > 0)), a.h, oy) * ry : INFINITY;
    float tz = sz ? fmaf((float)(iz + (sz > 0)), a.h, oz) * rz : INFINITY;
    const float dtx = a.h * fabsf(rx), dty = a.h * fabsf(ry), dtz = a.h * fabsf(rz);
    const float kx_per = fabsf(dx) * a.inv_h, ky_per = fabsf(dy) * a.inv_h, kz_per = fabsf(dz) * a.inv_h;
    // the ray leaves the grid at the last face of the first axis to run out
    const float t_grid =
        fminf(fminf(sx ? fmaf((float)(sx > 0 ? a.nx - 1 - ix : ix), dtx, tx) : INFINITY,
                    sy ? fmaf((float)(sy > 0 ? a.ny - 1 - iy : iy), dty, ty) : INFINITY),
              sz ? fmaf((float)(sz > 0 ? a.nz - 1 - iz : iz), dtz, tz) : INFINITY);
    const int nx = a.nx, ny = a.ny;
    int lin = (iz * ny + iy) * nx + ix;
    float t = 0.0f, sum = 0.0f;
    const int max_steps = a.nx + a.ny + a.nz + 3;
    for (int it = 0; it < max_steps; ++it) {
      const int m = __ldg(a.mat + lin);
      const int D = __ldg(a.skip + lin);
      const float e = (float)(D - 1);
      const float cx = fmaf(e, dtx, tx), cy = fmaf(e, dty, ty), cz = fmaf(e, dtz, tz);
      const float tc = fminf(fminf(fminf(cx, cy), cz), t_grid);
      sum = fmaf(mu_total<float>(c0, c1, c2, m, en), fmaxf(tc - t, 0.0f), sum);
      t = fmaxf(t, tc);
      if (tc >= t_grid) break;
      // faces crossed on each axis up to tc: all D on the axis that leaves
      // the cube, floor((tc - t_axis) / step) + 1 on the others
      const int kx = cx == tc ? D : (tx <= tc ? min((int)((tc - tx) * kx_per) + 1, D) : 0);
      const int ky = cy == tc ? D : (ty <= tc ? min((int)((tc - ty) * ky_per) + 1, D) : 0);
      const int kz = cz == tc ? D : (tz <= tc ? min((int)((tc - tz) * kz_per) + 1, D) : 0);
      ix += sx * kx;
      iy += sy * ky;
      iz += sz * kz;
      if ((unsigned)ix >= (unsigned)a.nx || (unsigned)iy >= (unsigned)a.ny || (unsigned)iz >= (unsigned)a.nz) break;
      tx = fmaf((float)kx, dtx, tx);
      ty = fmaf((float)ky, dty, ty);
      tz = fmaf((float)kz, dtz, tz);
      lin = (iz * ny + iy) * nx + ix;
    }
    return __expf(-sum);
  }
  int ix = voxel_index<T>(px, a.hx, a.h, a.inv_h, a.hx_h, a.nx);
  int iy = voxel_index<T>(py, a.hy, a.h, a.inv_h, a.hy_h, a.ny);
  int iz = voxel_index<T>(pz, a.hz, a.h, a.inv_h, a.hz_h, a.nz);
  const int sx = dx > (T)0 ? 1 : (dx < (T)0 ? -1 : 0);
  const int sy = dy > (T)0 ? 1 : (dy < (T)0 ? -1 : 0);
  const int sz = dz > (T)0 ? 1 : (dz < (T)0 ? -1 : 0);
  // distance along the ray to the next face on one axis
  auto face = [&](int i, int s, T half, T p, T d) -> T {
    if (s == 0) return (T)INFINITY;
    const T b = -half + (T)(i + (s > 0 ? 1 : 0)) * a.h;
    return (b - p) / d;
  };
  T tx = face(ix, sx, a.hx, px, dx), ty = face(iy, sy, a.hy, py, dy), tz = face(iz, sz, a.hz, pz, dz);
  T t = (T)0, sum = (T)0;
  const int max_steps = a.nx + a.ny + a.nz + 3;
  for (int it = 0; it < max_steps; ++it) {
    const int m = __ldg(a.mat + ((size_t)iz * a.ny + iy) * a.nx + ix);
    int ax = 0;
    T t1 = tx;
    if (ty < t1) { ax = 1; t1 = ty; }
    if (tz < t1) { ax = 2; t1 = tz; }
    if (t1 > t) {
      sum += mu_total<T>(c0, c1, c2, m, en) * (t1 - t);
      t = t1;
    }
    if (ax == 0) {
      ix += sx;
      if (ix < 0 || ix >= a.nx) break;
      tx = face(ix, sx, a.hx, px, dx);
    } else if (ax == 1) {
      iy += sy;
      if (iy < 0 || iy >= a.ny) break;
      ty = face(iy, sy, a.hy, py, dy);
    } else {
      iz += sz;
      if (iz < 0 || iz >= a.nz) break;
      tz = face(iz, sz, a.hz, pz, dz);
    }
  }
  if constexpr (is_dbl<T>()) return exp(-sum);
  else return __expf(-sum);
}

// Klein-Nishina angular density of the scattered direction per steradian,
// (dsigma/dOmega) / sigma_KN, dsigma/dOmega = (r_e^2/2) eps^2 (eps + 1/eps -
// sin^2 theta), eps = 1/(1 + alpha (1 - cos theta)).
template <typename T> __device__ __forceinline__ T kn_pdf_sr(T e, T mu, const Energy<T> &en) {
  if constexpr (is_dbl<T>()) {
    const double alpha = e / kMec2;
    const double eps = 1.0 / (1.0 + alpha * (1.0 - mu));
    const double dsig = 0.5 * kRe * kRe * (eps * eps) * (eps + 1.0 / eps - (1.0 - mu * mu));
    return dsig / en.sig;
  } else {
    const float den = 1.0f + e * (float)(1.0 / kMec2) * (1.0f - mu);
    const float eps = __fdividef(1.0f, den);
    const float dsig = (float)(0.5 * kRe * kRe) * (eps * eps) * (eps + den - (1.0f - mu * mu));
    return dsig / en.sig;
  }
}

// The forced copy of record r towards view k: a direction uniform in the
// collimator's acceptance cone about the view's normal, drawn from the
// copy's own Philox block (counter (k, 1 + n, h_lo, h_hi)), weighted by
// the survival at the interaction, the angular probability of that
// direction, the collimator's open fraction and the transmission to the
// grid boundary, then binned like an analog detection.
template <typename T>
__device__ __forceinline__ void fd_copy(const TArgs<T> &a, const FdRec<T> &r, int k, const T *c0, const T *c1,
                                        const T *c2, const float *sig_tab) {
  uint32_t w0 = (uint32_t)k, w1 = 1u + r.n, w2 = (uint32_t)r.h, w3 = (uint32_t)(r.h >> 32);
  philox_rounds(w0, w1, w2, w3, a.rk);
  const T u0 = uniform<T>(w0), u1 = uniform<T>(w1), u2 = uniform<T>(w2), u3 = uniform<T>(w3);
  const T ck = a.view_cs[2 * k], sk = a.view_cs[2 * k + 1];
  T ct, st;
  if constexpr (is_dbl<T>()) {
    ct = 1.0 - u0 * (1.0 - a.cos_max);
    st = sqrt0<double>(1.0 - ct * ct);
  } else {
    // 1 - cos is a few 1e-3 at most: sin^2 = (1 - cos)(1 + cos) keeps float's
    // relative precision where 1 - cos^2 would cancel
    const float om = u0 * a.one_m_cos_max;
    ct = 1.0f - om;
    st = sqrt0<float>(om * (2.0f - om));
  }
  T cph, sph;
  cos_sin_2pi<T>(u1, cph, sph);
  const T dx = ct * ck - st * cph * sk, dy = ct * sk + st * cph * ck, dz = st * sph;
  if (!(a.ratio * st < ct)) return;
  const T x = a.ratio * st / ct;
  const T pass = (T)(2.0 / kPi) * (acos(x) - x * sqrt0<T>((T)1 - x * x));
  T ang, e1;
  if (r.n == 0) {
    ang = a.omega_4pi;
    e1 = r.e;
  } else {
    const T mu_s = r.d[0] * dx + r.d[1] * dy + r.d[2] * dz;
    if constexpr (is_dbl<T>()) {
      const double eps = 1.0 / (1.0 + (r.e / kMec2) * (1.0 - mu_s));
      e1 = eps * r.e;
    } else {
      e1 = __fdividef(r.e, 1.0f + r.e * (float)(1.0 / kMec2) * (1.0f - mu_s));
    }
    if (e1 < a.e_low) return;
    Energy<T> en;
    en.set(r.e, a, sig_tab);
    ang = a.omega * kn_pdf_sr<T>(r.e, mu_s, en);
  }
  const T wt = r.keep * ang * pass * transmission<T>(a, r.p[0], r.p[1], r.p[2], dx, dy, dz, e1, c0, c1, c2, sig_tab);
  const long long q = __double2ll_rn((double)wt * kFdScale);
  if (q <= 0) return;
  const T t = (a.plane - (r.p[0] * ck + r.p[1] * sk)) / ct;
  const T qx = r.p[0] + t * dx, qy = r.p[1] + t * dy, qz = r.p[2] + t * dz;
  T au = -qx * sk + qy * ck;
  T bv = qz;
  T rr;
  if constexpr (is_dbl<T>()) rr = sqrt(-2.0 * log(u2));
  else rr = sqrt0<float>(-2.0f * __logf(u2));
  T cb, sb;
  cos_sin_2pi<T>(u3, cb, sb);
  au += a.sigma * (rr * cb);
  bv += a.sigma * (rr * sb);
  const T fu = floor(au / a.bin + a.half_bu);
  const T fv = floor(bv / a.bin + a.half_bv);
  if (!(fu >= (T)0 && fu < (T)a.bins_u && fv >= (T)0 && fv < (T)a.bins_v)) return;
  const uint64_t row = ((uint64_t)k * a.bins_v + (uint64_t)fv) * a.bins_u + (uint64_t)fu;
  const uint64_t v = r.h % a.n_vox;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned long long base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(a.cursor, (unsigned long long)g.size());
  base = g.shfl(base, 0);
  const unsigned long long idx = base + g.thread_rank();
  if (idx < a.capacity) {
    a.events[idx] = (unsigned long long)(v * a.n_rows + row);
    a.weights[idx] = (unsigned long long)q;
  }
}

// One thread per (queued interaction, view), views fastest.
template <typename T>
__global__ void __launch_bounds__(256) fd_kernel(const __grid_constant__ TArgs<T> a) {
  __shared__ T s_c0[256], s_c1[256], s_c2[256];
  __shared__ float s_sig[kSigTab];
  for (int m = threadIdx.x; m < a.n_mat; m += blockDim.x) {
    s_c0[m] = a.coef[3 * m];
    s_c1[m] = a.coef[3 * m + 1];
    s_c2[m] = a.coef[3 * m + 2];
  }
  if (!is_dbl<T>())
    for (int i = threadIdx.x; i < kSigTab; i += blockDim.x) s_sig[i] = a.sig_tab[i];
  __syncthreads();
  const unsigned long long n_q = *a.esc_cursor < a.esc_capacity ? *a.esc_cursor : a.esc_capacity;
  const unsigned long long total = n_q * (unsigned long long)a.n_views;
  const FdRec<T> *q = static_cast<const FdRec<T> *>(a.esc);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long ri = i / (unsigned long long)a.n_views;
    const int k = (int)(i - ri * (unsigned long long)a.n_views);
    fd_copy<T>(a, q[ri], k, s_c0, s_c1, s_c2, s_sig);
  }
}

// Compton sampler alone (verification).
template <typename T>
__global__ void debug_kn_kernel(const __grid_constant__ TArgs<T> a, T e, uint64_t n, double *cos_out, double *eps_out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    KStream st;
    st.init(i);
    KRng rng{st, a.rk};
    T mu = 0, eps = 0;
    compton<T>(rng, e, mu, eps);
    cos_out[i] = (double)mu;
    eps_out[i] = (double)eps;
  }
}

// Woodcock flight alone (verification): photons from p0 along d, counts
// those that leave the grid without a real collision.
template <typename T>
__global__ void debug_beam_kernel(const __grid_constant__ TArgs<T> a, T p0x, T p0y, T p0z, T dx, T dy, T dz, T e,
                                  uint64_t n, unsigned long long *through) {
  __shared__ T s_c0[256], s_c1[256], s_c2[256];
  __shared__ float s_sig[kSigTab];
  for (int m = threadIdx.x; m < a.n_mat; m += blockDim.x) {
    s_c0[m] = a.coef[3 * m];
    s_c1[m] = a.coef[3 * m + 1];
    s_c2[m] = a.coef[3 * m + 2];
  }
  if (!is_dbl<T>())
    for (int i = threadIdx.x; i < kSigTab; i += blockDim.x) s_sig[i] = a.sig_tab[i];
  __syncthreads();
  Energy<T> en;
  en.set(e, a, s_sig);
  unsigned long long mine = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!(a.mu_maj > (T)0)) { mine += 1; continue; }
    KStream st;
    st.init(i);
    T px = p0x, py = p0y, pz = p0z;
    for (uint32_t s = 0; s < kStepCap; ++s) {
      const T l = flight<T>(uniform<T>(st.word(a.rk)), a);
      const T qx = px + l * dx, qy = py + l * dy, qz = pz + l * dz;
      if (!(qx >= -a.hx && qx < a.hx && qy >= -a.hy && qy < a.hy && qz >= -a.hz && qz < a.hz)) { mine += 1; break; }
      px = qx; py = qy; pz = qz;
      const int ix = voxel_index<T>(px, a.hx, a.h, a.inv_h, a.hx_h, a.nx);
      const int iy = voxel_index<T>(py, a.hy, a.h, a.inv_h, a.hy_h, a.ny);
      const int iz = voxel_index<T>(pz, a.hz, a.h, a.inv_h, a.hz_h, a.nz);
      const int m = a.mat[((size_t)iz * a.ny + iy) * a.nx + ix];
      if (uniform<T>(st.word(a.rk)) * a.mu_maj < mu_total<T>(s_c0, s_c1, s_c2, m, en)) break;
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

inline void round_keys(uint32_t key0, uint32_t key1, uint32_t rk[20]) {
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = key0 + (uint32_t)r * 0x9E3779B9u;
    rk[2 * r + 1] = key1 + (uint32_t)r * 0xBB67AE85u;
  }
}

// float path: sigma_KN tabulated at E_low + i (E0 - E_low) / (kSigTab - 1)
inline void host_sigma_table(const TransportSetup &ts, std::vector<float> &tab) {
  const double el = host_e_low(ts), de = (ts.e0 - el) / (kSigTab - 1);
  tab.resize(kSigTab);
  for (int i = 0; i < kSigTab; ++i) tab[i] = (float)host_sigma_kn(el + i * de);
}

template <typename T> void make_targs(const TransportSetup &ts, TArgs<T> &a) {
  std::memset(&a, 0, sizeof(a));
  a.coef = std::is_same<T, double>::value ? (const T *)(const void *)ts.coef_d_dev
                                          : (const T *)(const void *)ts.coef_f_dev;
  a.mat = ts.material_dev;
  a.view_cs = std::is_same<T, double>::value ? (const T *)(const void *)ts.view_cs_dev
                                             : (const T *)(const void *)ts.view_cs_f_dev;
  a.sig_tab = ts.sig_tab_dev;
  a.skip = ts.skip_dev;
  round_keys(ts.key0, ts.key1, a.rk);
  a.nx = ts.nx; a.ny = ts.ny; a.nz = ts.nz; a.n_mat = ts.n_mat;
  a.h = (T)ts.h;
  a.hx = (T)(0.5 * ts.nx * ts.h);
  a.hy = (T)(0.5 * ts.ny * ts.h);
  a.hz = (T)(0.5 * ts.nz * ts.h);
  a.inv_h = (T)(1.0 / ts.h);
  a.hx_h = (T)(0.5 * ts.nx);
  a.hy_h = (T)(0.5 * ts.ny);
  a.hz_h = (T)(0.5 * ts.nz);
  const double maj = host_majorant(ts);
  a.mu_maj = (T)maj;
  a.inv_mu_maj = (T)(maj > 0.0 ? 1.0 / maj : 0.0);
  a.e0 = (T)ts.e0;
  const double el = host_e_low(ts);
  a.e_low = (T)el;
  a.inv_de = (T)((kSigTab - 1) / (ts.e0 - el));
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
  a.events = ts.events; a.capacity = ts.capacity; a.cursor = ts.cursor; a.fates = ts.fates;
  a.records = ts.records;
  a.primary_only = ts.primary_only;
  a.t_coll = kWaitCollide;
  a.t_emit = kWaitEmit;
  a.esc = ts.esc;
  a.esc_capacity = ts.esc_capacity;
  a.esc_cursor = ts.esc_cursor;
  a.weights = ts.weights;
  const double cos_max = 1.0 / std::sqrt(1.0 + tan_max * tan_max);
  const double omega = 2.0 * kPi * (1.0 - cos_max);
  a.cos_max = (T)cos_max;
  a.omega = (T)omega;
  a.omega_4pi = (T)(omega / (4.0 * kPi));
  a.one_m_cos_max = (T)(1.0 - cos_max);
  const double band = tan_max / std::sqrt(1.0 + tan_max * tan_max);
  a.forced_dir = ts.forced_dir;
  a.band = (T)band;
  a.q_dir = (unsigned long long)std::llrint(band * kFdScale);
}

template <typename T> int launch_transport_t(const TransportSetup &ts, cudaStream_t s) {
  TArgs<T> a;
  make_targs<T>(ts, a);
  if (ts.count == 0) return MC_OK;
  if (ts.forced && !is_dbl<T>() && !ts.skip_dev) {
    set_error("float forced detection needs the plan's distance map");
    return MC_EINVAL;
  }
  const int threads = 256;
  int per_sm = 0;
  if (ts.forced) {
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_kernel<T, false, true>, threads, 0));
  } else if (ts.records) {
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_kernel<T, true>, threads, 0));
  } else {
    MCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, transport_kernel<T, false>, threads, 0));
  }
  if (per_sm < 1) per_sm = 1;
  const int64_t full = (int64_t)device_sm_count() * per_sm;
  const int64_t need = (int64_t)((ts.count + threads - 1) / threads);
  const int grid = (int)(need < full ? need : full);
  a.stride = (uint64_t)grid * threads;
  {
    const uint32_t sm = (uint32_t)(a.stride % a.n_vox);
    a.step_v[0] = sm % (uint32_t)ts.nx;
    a.step_v[1] = (sm / (uint32_t)ts.nx) % (uint32_t)ts.ny;
    a.step_v[2] = sm / ((uint32_t)ts.nx * (uint32_t)ts.ny);
  }
  if (ts.forced) { count_launch(); transport_kernel<T, false, true><<<grid, threads, 0, s>>>(a); }
  else if (ts.records) { count_launch(); transport_kernel<T, true><<<grid, threads, 0, s>>>(a); }
  else { count_launch(); transport_kernel<T, false><<<grid, threads, 0, s>>>(a); }
  MCS_LAUNCHED();
  if (ts.ev_mid) MCS_CUDA(cudaEventRecord(ts.ev_mid, s));
  const int dgrid = device_sm_count() * 8;
  if (ts.forced) { count_launch(); fd_kernel<T><<<dgrid, 256, 0, s>>>(a); }
  else if (ts.records) { count_launch(); detect_kernel<T, true><<<dgrid, 256, 0, s>>>(a); }
  else { count_launch(); detect_kernel<T, false><<<dgrid, 256, 0, s>>>(a); }
  MCS_LAUNCHED();
  return MC_OK;
}

template <typename T>
int launch_debug_kn_t(double e_kev, uint64_t seed, uint64_t n, double *cos_dev, double *eps_dev, cudaStream_t s) {
  if (n == 0) return MC_OK;
  TArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  round_keys((uint32_t)seed, (uint32_t)(seed >> 32), a.rk);
  const int threads = 256;
  const int64_t need = (int64_t)((n + threads - 1) / threads);
  const int grid = (int)(need < 4096 ? need : 4096);
  count_launch(); debug_kn_kernel<T><<<grid, threads, 0, s>>>(a, (T)e_kev, n, cos_dev, eps_dev);
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
