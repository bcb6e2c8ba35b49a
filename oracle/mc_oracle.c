/*
 * mc_oracle.c -- plain, slow FP64 CPU oracle for analog Monte Carlo SPECT
 * system-matrix transport.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark do.  It shares no code, header or constant table with
 * the CUDA implementation: every definition below is written out again from
 * the transport contract stated in the comments.
 *
 * What it computes (paper Sec. 2 and Sec. 5.1):
 *   - each source photon (a "history") is followed from its emission until it
 *     is absorbed, drops below the energy window or escapes the phantom,
 *     sampling every step from cross-sections (Sec. 2);
 *   - an escaping photon that passes the parallel-hole collimator of a view
 *     is binned on that view's detector (Sec. 3, "the collimator allows only
 *     the photons impinging on the front face of the detector");
 *   - every detection is a tally event (row j, column v); counting the events
 *     estimates T_ij of Eq. (IMC), the probability that a photon from voxel i
 *     is detected in pixel j (Sec. 5.1).
 *
 * Readings of the paper (it gives physics only in words):
 *   R1  Philox4x32-10 counter-based streams keyed by (seed, history id).
 *   R2  Woodcock (delta) tracking over one majorant mu_maj.
 *   R3  mu(m,E) = 0.1 * rho_m * (N_A (Z/A)_m sigma_KN(E) + k Z_eff^4 / E^3)
 *       in 1/mm (E in keV); sigma_KN = closed-form Klein-Nishina total.
 *   R4  Compton scattering by plain rejection on a uniform cos(theta); no
 *       Rayleigh scattering; ideal energy resolution, so a photon leaves the
 *       window only by dropping below (1 - w/2) E0.
 *   R5  ideal parallel-hole collimator: an escaping photon at angle psi to a
 *       view's axis passes with probability f(x) = (2/pi)(acos x - x sqrt(1-x^2)),
 *       x = (L/d) tan psi, the overlap fraction of the two ends of a hole.
 *   R6  Gaussian intrinsic blur (FWHM) by Box-Muller on two draws.
 *   R7  forced detection (the variance-reduction technique of the paper's
 *       Sec. 4 on VRT: a copy of the photon is forced to the detector at
 *       each interaction location and weighted by the probability of not
 *       being absorbed there, of leaving in a direction the collimator
 *       passes, and of crossing the medium unabsorbed).  Interaction
 *       locations are the emission point (n = 0) and every real collision
 *       (n = 1, 2, ...).  For each view k the copy's direction is drawn
 *       uniformly in the cone of directions the collimator can pass
 *       (tan(psi) < d/L about the view's normal) from its own stream
 *       block, counter (k, 1 + n, h_lo, h_hi), which the analog stream never
 *       reaches (its block index stays below 2^32).  Weight:
 *         emission:  Omega_c / (4 pi) * f(x) * T(p, d, E0)
 *         collision: (1 - mu_pe/mu) * Omega_c * p_KN(cos theta_s | E)
 *                    * f(x) * T(p, d, E')   (0 if E' = eps E < E_low)
 *       with Omega_c the cone's solid angle, p_KN the Klein-Nishina
 *       angular density per steradian, T the exact transmission along the
 *       ray to the grid boundary.  The copy is binned like an analog
 *       detection (crystal hit, Gaussian blur on the block's last two
 *       words); the analog photon itself is no longer detected.  Weights
 *       are tallied in fixed point, q = rint(w 2^48), so that sums are
 *       exact integers whatever their order.
 *   R8  forced direction (same section): the emission direction is drawn
 *       only from the band |d_z| < sin(psi_max), psi_max = atan(d/L), the
 *       directions from which some view's collimator can be reached
 *       (cos(theta) uniform in the band, same draws), and every detection
 *       carries the band's share of the sphere, w = sin(psi_max).  Exact
 *       for photons that reach the camera unscattered; scattered photons
 *       from emissions outside the band are not simulated, so it is offered
 *       with the primary-only tally only.
 *
 * Precision: every floating-point value is an IEEE double.  Build with
 * -ffp-contract=off so that no multiply-add is fused and the results are the
 * same on every host.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* physical constants (CODATA 2018)                                          */
/* ------------------------------------------------------------------------ */
#define ORC_AVOGADRO 6.02214076e23      /* 1/mol */
#define ORC_RE_CM 2.8179403262e-13      /* classical electron radius, cm */
#define ORC_MEC2_KEV 510.99895          /* electron rest energy, keV */
#define ORC_PI 3.14159265358979323846

/* transport caps: a history that reaches them ends with fate CAP */
#define ORC_STEP_CAP 1000000u
#define ORC_TRIAL_CAP 10000u

enum { ORC_FATE_ABSORBED = 0, ORC_FATE_BELOW_WINDOW = 1, ORC_FATE_ESCAPE = 2, ORC_FATE_CAP = 3 };
#define ORC_MAX_REC_EVENTS 4

/* The problem description handed in by the Python side of the oracle. */
typedef struct {
  int32_t nx, ny, nz;
  double voxel_mm;
  const uint8_t *material; /* nz*ny*nx, x fastest */
  int32_t n_materials;
  const double *rho, *z_over_a, *z_eff;
  int32_t n_views;
  double start_deg, arc_deg;
  int32_t n_bins_u, n_bins_v;
  double bin_mm;
  double radius_mm; /* distance of the collimator front face from the axis */
  double hole_len_mm, hole_diam_mm;
  double fwhm_mm;
  double e0_kev, window_frac, photo_k;
  int32_t primary_only; /* 1: tally only photons that never scattered */
  int32_t forced_detection; /* 1: R7 forced detection instead of analog detection */
  int32_t forced_direction; /* 1: R8 forced emission direction (with primary_only) */
} orc_problem;

typedef struct {
  uint8_t fate, n_events;
  uint16_t pad;
  uint32_t n_virtual, n_real, n_compton, n_draws;
  uint32_t pad2;
  double e_final_kev;
  int32_t event_row[ORC_MAX_REC_EVENTS];
} orc_record;

/* ------------------------------------------------------------------------ */
/* R1: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3).           */
/* One round maps (c0,c1,c2,c3) with multipliers M0, M1 to                    */
/*   (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0));                */
/* the key is bumped by the Weyl constants between rounds.                   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The stream of history h: words 0..3 of block 0 (counter (0,0,h_lo,h_hi)),
 * then block 1, ...; one draw = one word; u = (w + 0.5) 2^-32 in (0,1). */
typedef struct {
  uint32_t key[2];
  uint64_t history;
  uint64_t block;
  uint32_t word[4];
  int next;
  uint32_t n_draws;
} orc_stream;

static void stream_init(orc_stream *s, uint64_t seed, uint64_t history) {
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->history = history;
  s->block = 0;
  s->next = 4;
  s->n_draws = 0;
}

static double draw(orc_stream *s) {
  if (s->next == 4) {
    uint32_t ctr[4] = {(uint32_t)s->block, (uint32_t)(s->block >> 32), (uint32_t)s->history,
                       (uint32_t)(s->history >> 32)};
    orc_philox4x32_10(ctr, s->key, s->word);
    s->block += 1;
    s->next = 0;
  }
  uint32_t w = s->word[s->next++];
  s->n_draws += 1;
  return ((double)w + 0.5) * (1.0 / 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* R3: cross-sections                                                        */
/* ------------------------------------------------------------------------ */

/* Klein-Nishina total cross-section per electron, cm^2 (Klein & Nishina
 * 1929; e.g. Evans, "The Atomic Nucleus", ch. 23). */
double orc_sigma_kn_cm2(double e_kev) {
  double a = e_kev / ORC_MEC2_KEV;
  double t = 1.0 + 2.0 * a;
  double l = log(t);
  double term1 = (1.0 + a) / (a * a) * (2.0 * (1.0 + a) / t - l / a);
  double term2 = l / (2.0 * a);
  double term3 = (1.0 + 3.0 * a) / (t * t);
  return 2.0 * ORC_PI * ORC_RE_CM * ORC_RE_CM * (term1 + term2 - term3);
}

/* Photoelectric attenuation of material m at energy e, 1/mm. */
static double mu_photo(const orc_problem *pb, int m, double e_kev) {
  double z = pb->z_eff[m];
  double z4 = (z * z) * (z * z);
  return 0.1 * pb->rho[m] * (pb->photo_k * z4 / (e_kev * e_kev * e_kev));
}

/* Total attenuation of material m at energy e, 1/mm. */
double orc_mu_total(const orc_problem *pb, int m, double e_kev) {
  double z = pb->z_eff[m];
  double z4 = (z * z) * (z * z);
  double compton = ORC_AVOGADRO * pb->z_over_a[m] * orc_sigma_kn_cm2(e_kev);
  double photo = pb->photo_k * z4 / (e_kev * e_kev * e_kev);
  return 0.1 * pb->rho[m] * (compton + photo);
}

/* Lower edge of the energy window. */
static double e_low(const orc_problem *pb) { return (1.0 - 0.5 * pb->window_frac) * pb->e0_kev; }

/* Majorant: the largest mu over the material table at the window's lower
 * edge.  Both terms of mu fall with E, so it bounds mu for every energy a
 * tracked photon can have. */
double orc_majorant(const orc_problem *pb) {
  double el = e_low(pb), best = 0.0;
  for (int m = 0; m < pb->n_materials; ++m) {
    double mu = orc_mu_total(pb, m, el);
    if (mu > best) best = mu;
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* geometry: grid centred on the origin, box [-n h/2, n h/2) on each axis     */
/* ------------------------------------------------------------------------ */
static int inside_box(const orc_problem *pb, const double p[3]) {
  double hx = 0.5 * pb->nx * pb->voxel_mm, hy = 0.5 * pb->ny * pb->voxel_mm, hz = 0.5 * pb->nz * pb->voxel_mm;
  return p[0] >= -hx && p[0] < hx && p[1] >= -hy && p[1] < hy && p[2] >= -hz && p[2] < hz;
}

static int axis_index(double x, int n, double h) {
  double half = 0.5 * n * h;
  int i = (int)floor((x + half) / h);
  return i > n - 1 ? n - 1 : i;
}

static int material_at(const orc_problem *pb, const double p[3]) {
  int i = axis_index(p[0], pb->nx, pb->voxel_mm);
  int j = axis_index(p[1], pb->ny, pb->voxel_mm);
  int k = axis_index(p[2], pb->nz, pb->voxel_mm);
  return pb->material[((int64_t)k * pb->ny + j) * pb->nx + i];
}

/* ------------------------------------------------------------------------ */
/* one history                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t n_steps, n_virtual, n_real, n_compton;
} orc_counts;

/* R2: fly from p along d until the next real collision.  Returns 0 with p
 * moved to the collision site, 1 if the flight leaves the box (p is left at
 * its pre-flight value), 2 if the step cap is reached. */
static int woodcock_flight(const orc_problem *pb, orc_stream *s, double p[3], const double d[3], double e_kev,
                           double mu_maj, orc_counts *c, int *m_out, double *mu_out) {
  if (!(mu_maj > 0.0)) return 1;
  for (;;) {
    if (c->n_steps >= ORC_STEP_CAP) return 2;
    c->n_steps += 1;
    double step = -log(draw(s)) / mu_maj;
    double q[3] = {p[0] + step * d[0], p[1] + step * d[1], p[2] + step * d[2]};
    if (!inside_box(pb, q)) return 1;
    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
    int m = material_at(pb, p);
    double mu = orc_mu_total(pb, m, e_kev);
    if (draw(s) * mu_maj < mu) {
      c->n_real += 1;
      *m_out = m;
      *mu_out = mu;
      return 0;
    }
    c->n_virtual += 1;
  }
}

/* R4: Klein-Nishina polar angle by rejection.  Returns 0 and sets cos(theta)
 * and eps = E'/E, or 1 if the trial cap is reached. */
static int compton_sample(orc_stream *s, double e_kev, double *mu_c, double *eps_out) {
  double alpha = e_kev / ORC_MEC2_KEV;
  for (uint32_t t = 0; t < ORC_TRIAL_CAP; ++t) {
    double mu = 2.0 * draw(s) - 1.0;
    double eps = 1.0 / (1.0 + alpha * (1.0 - mu));
    double f = 0.5 * eps * eps * (eps + 1.0 / eps - (1.0 - mu * mu));
    if (draw(s) < f) {
      *mu_c = mu;
      *eps_out = eps;
      return 0;
    }
  }
  return 1;
}

/* New direction after a deflection by polar cosine mu and azimuth phi about
 * the old direction d (the usual frame rotation of photon transport codes). */
void orc_rotate(double d[3], double mu, double phi) {
  double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  double cp = cos(phi), sp = sin(phi);
  double u = d[0], v = d[1], w = d[2];
  double nu, nv, nw;
  if (fabs(w) < 0.99999) {
    double r = sqrt(1.0 - w * w);
    nu = mu * u + st * (u * w * cp - v * sp) / r;
    nv = mu * v + st * (v * w * cp + u * sp) / r;
    nw = mu * w - st * cp * r;
  } else {
    nu = st * cp;
    nv = st * sp;
    nw = (w >= 0.0 ? mu : -mu);
  }
  double n = sqrt(nu * nu + nv * nv + nw * nw);
  d[0] = nu / n; d[1] = nv / n; d[2] = nw / n;
}

/* R5 + R6: offer an escaping photon (p inside the box, direction d) to every
 * view in ascending order; calls emit(row) for each detection. */
typedef void (*orc_emit_fn)(void *ctx, int32_t row);

static void detect(const orc_problem *pb, orc_stream *s, const double p[3], const double d[3], orc_emit_fn emit,
                   void *ctx) {
  double ratio = pb->hole_len_mm / pb->hole_diam_mm;
  double sigma = pb->fwhm_mm / (2.0 * sqrt(2.0 * log(2.0)));
  double plane = pb->radius_mm + pb->hole_len_mm;
  for (int k = 0; k < pb->n_views; ++k) {
    double th = (pb->start_deg + k * (pb->arc_deg / pb->n_views)) * (ORC_PI / 180.0);
    double ck = cos(th), sk = sin(th);
    double c = d[0] * ck + d[1] * sk;
    if (!(c > 0.0)) continue;
    double st = sqrt(fmax(0.0, 1.0 - c * c));
    if (!(ratio * st < c)) continue;
    double x = ratio * st / c;
    double pass = (2.0 / ORC_PI) * (acos(x) - x * sqrt(1.0 - x * x));
    if (!(draw(s) < pass)) continue;
    double t = (plane - (p[0] * ck + p[1] * sk)) / c;
    double q[3] = {p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2]};
    double a = -q[0] * sk + q[1] * ck;
    double b = q[2];
    double u1 = draw(s), u2 = draw(s);
    double r = sqrt(-2.0 * log(u1));
    a += sigma * (r * cos(2.0 * ORC_PI * u2));
    b += sigma * (r * sin(2.0 * ORC_PI * u2));
    double fu = floor(a / pb->bin_mm + 0.5 * pb->n_bins_u);
    double fv = floor(b / pb->bin_mm + 0.5 * pb->n_bins_v);
    if (fu < 0.0 || fu >= pb->n_bins_u || fv < 0.0 || fv >= pb->n_bins_v) continue;
    int32_t row = (int32_t)(((int64_t)k * pb->n_bins_v + (int64_t)fv) * pb->n_bins_u + (int64_t)fu);
    emit(ctx, row);
  }
}

/* ------------------------------------------------------------------------ */
/* R7: forced detection                                                      */
/* ------------------------------------------------------------------------ */
#define ORC_FD_SCALE 281474976710656.0 /* 2^48 */

/* Klein-Nishina angular density of the scattered direction, per steradian:
 * (dsigma/dOmega) / sigma_KN with dsigma/dOmega = (r_e^2 / 2) eps^2
 * (eps + 1/eps - sin^2 theta), eps = 1 / (1 + alpha (1 - cos theta)). */
double orc_kn_pdf_sr(double e_kev, double mu) {
  double alpha = e_kev / ORC_MEC2_KEV;
  double eps = 1.0 / (1.0 + alpha * (1.0 - mu));
  double dsig = 0.5 * ORC_RE_CM * ORC_RE_CM * (eps * eps) * (eps + 1.0 / eps - (1.0 - mu * mu));
  return dsig / orc_sigma_kn_cm2(e_kev);
}

/* exp(-integral of mu(E) along the ray p + t d, t >= 0, up to the grid
 * boundary), by visiting the voxels the ray crosses in order (a 3-D DDA:
 * the next voxel is across the nearest of the three next faces, ties to
 * the lowest axis).  p must be inside the box; d a unit vector. */
double orc_transmission(const orc_problem *pb, const double p[3], const double d[3], double e_kev) {
  int n[3] = {pb->nx, pb->ny, pb->nz};
  double h = pb->voxel_mm;
  double mu_m[256];
  for (int m = 0; m < pb->n_materials; ++m) mu_m[m] = orc_mu_total(pb, m, e_kev);
  int idx[3], step[3];
  double tn[3];
  for (int a = 0; a < 3; ++a) {
    double half = 0.5 * n[a] * h;
    idx[a] = axis_index(p[a], n[a], h);
    if (d[a] > 0.0) {
      step[a] = 1;
      tn[a] = ((-half + (idx[a] + 1) * h) - p[a]) / d[a];
    } else if (d[a] < 0.0) {
      step[a] = -1;
      tn[a] = ((-half + idx[a] * h) - p[a]) / d[a];
    } else {
      step[a] = 0;
      tn[a] = INFINITY;
    }
  }
  /* a direction with no finite non-zero component never leaves the grid:
     the line integral is undefined */
  if (step[0] == 0 && step[1] == 0 && step[2] == 0) return NAN;
  double t = 0.0, sum = 0.0;
  for (;;) {
    int m = pb->material[((int64_t)idx[2] * pb->ny + idx[1]) * pb->nx + idx[0]];
    int a = 0;
    if (tn[1] < tn[a]) a = 1;
    if (tn[2] < tn[a]) a = 2;
    double t1 = tn[a];
    if (t1 > t) {
      sum += mu_m[m] * (t1 - t);
      t = t1;
    }
    idx[a] += step[a];
    if (idx[a] < 0 || idx[a] >= n[a]) break;
    double half = 0.5 * n[a] * h;
    tn[a] = ((-half + (idx[a] + (step[a] > 0 ? 1 : 0)) * h) - p[a]) / d[a];
  }
  return exp(-sum);
}

typedef void (*orc_emit_w_fn)(void *ctx, int32_t row, int64_t q);

/* The forced copies of interaction n of history h (at p, energy e, incoming
 * direction d_in; p_keep = 1 - mu_pe/mu at a collision, 1 at emission). */
static void fd_point(const orc_problem *pb, uint64_t seed, uint64_t h, uint32_t n, const double p[3],
                     const double d_in[3], double e, double p_keep, int emission, orc_emit_w_fn emit, void *ctx) {
  double ratio = pb->hole_len_mm / pb->hole_diam_mm;
  double sigma = pb->fwhm_mm / (2.0 * sqrt(2.0 * log(2.0)));
  double plane = pb->radius_mm + pb->hole_len_mm;
  double tan_max = pb->hole_diam_mm / pb->hole_len_mm;
  double cos_max = 1.0 / sqrt(1.0 + tan_max * tan_max);
  double omega = 2.0 * ORC_PI * (1.0 - cos_max);
  double elow = e_low(pb);
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int k = 0; k < pb->n_views; ++k) {
    uint32_t ctr[4] = {(uint32_t)k, 1u + n, (uint32_t)h, (uint32_t)(h >> 32)}, w[4];
    orc_philox4x32_10(ctr, key, w);
    double u0 = ((double)w[0] + 0.5) * (1.0 / 4294967296.0);
    double u1 = ((double)w[1] + 0.5) * (1.0 / 4294967296.0);
    double u2 = ((double)w[2] + 0.5) * (1.0 / 4294967296.0);
    double u3 = ((double)w[3] + 0.5) * (1.0 / 4294967296.0);
    double th = (pb->start_deg + k * (pb->arc_deg / pb->n_views)) * (ORC_PI / 180.0);
    double ck = cos(th), sk = sin(th);
    /* direction uniform in the acceptance cone about (ck, sk, 0) */
    double ct = 1.0 - u0 * (1.0 - cos_max);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double cph = cos(2.0 * ORC_PI * u1), sph = sin(2.0 * ORC_PI * u1);
    double d[3] = {ct * ck - st * cph * sk, ct * sk + st * cph * ck, st * sph};
    if (!(ratio * st < ct)) continue;
    double x = ratio * st / ct;
    double pass = (2.0 / ORC_PI) * (acos(x) - x * sqrt(1.0 - x * x));
    double ang, e1;
    if (emission) {
      ang = omega / (4.0 * ORC_PI);
      e1 = e;
    } else {
      double mu_s = d_in[0] * d[0] + d_in[1] * d[1] + d_in[2] * d[2];
      double eps = 1.0 / (1.0 + (e / ORC_MEC2_KEV) * (1.0 - mu_s));
      e1 = eps * e;
      if (e1 < elow) continue;
      ang = omega * orc_kn_pdf_sr(e, mu_s);
    }
    double wt = p_keep * ang * pass * orc_transmission(pb, p, d, e1);
    int64_t q = (int64_t)llrint(wt * ORC_FD_SCALE);
    if (q <= 0) continue;
    double t = (plane - (p[0] * ck + p[1] * sk)) / ct;
    double qp[3] = {p[0] + t * d[0], p[1] + t * d[1], p[2] + t * d[2]};
    double a = -qp[0] * sk + qp[1] * ck;
    double b = qp[2];
    double r = sqrt(-2.0 * log(u2));
    a += sigma * (r * cos(2.0 * ORC_PI * u3));
    b += sigma * (r * sin(2.0 * ORC_PI * u3));
    double fu = floor(a / pb->bin_mm + 0.5 * pb->n_bins_u);
    double fv = floor(b / pb->bin_mm + 0.5 * pb->n_bins_v);
    if (fu < 0.0 || fu >= pb->n_bins_u || fv < 0.0 || fv >= pb->n_bins_v) continue;
    int32_t row = (int32_t)(((int64_t)k * pb->n_bins_v + (int64_t)fv) * pb->n_bins_u + (int64_t)fu);
    emit(ctx, row, q);
  }
}

/* R8: half-width of the forced emission band in cos(theta) (= its share of
 * the sphere): sin(psi_max), tan(psi_max) = d/L. */
double orc_direction_band(const orc_problem *pb) {
  double tan_max = pb->hole_diam_mm / pb->hole_len_mm;
  return tan_max / sqrt(1.0 + tan_max * tan_max);
}

/* Follow history h to its end.  Fills rec (if not NULL) and calls emit. */
static void run_history(const orc_problem *pb, uint64_t seed, uint64_t h, double mu_maj, orc_record *rec,
                        orc_emit_fn emit, orc_emit_w_fn emit_w, void *ctx) {
  orc_stream s;
  stream_init(&s, seed, h);
  orc_counts c = {0, 0, 0, 0};
  int64_t n_vox = (int64_t)pb->nx * pb->ny * pb->nz;
  int64_t v = (int64_t)(h % (uint64_t)n_vox);
  int64_t vi = v % pb->nx, vj = (v / pb->nx) % pb->ny, vk = v / ((int64_t)pb->nx * pb->ny);
  double hv = pb->voxel_mm;
  double p[3];
  p[0] = ((double)vi + draw(&s)) * hv - 0.5 * pb->nx * hv;
  p[1] = ((double)vj + draw(&s)) * hv - 0.5 * pb->ny * hv;
  p[2] = ((double)vk + draw(&s)) * hv - 0.5 * pb->nz * hv;
  double ct = 2.0 * draw(&s) - 1.0;
  if (pb->forced_direction) ct = ct * orc_direction_band(pb);
  double phi = 2.0 * ORC_PI * draw(&s);
  double st = sqrt(fmax(0.0, 1.0 - ct * ct));
  double d[3] = {st * cos(phi), st * sin(phi), ct};
  double e = pb->e0_kev;
  double elow = e_low(pb);
  int fd = pb->forced_detection && emit_w;
  if (fd) fd_point(pb, seed, h, 0u, p, d, e, 1.0, 1, emit_w, ctx);
  int fate;
  for (;;) {
    int m;
    double mu;
    int r = woodcock_flight(pb, &s, p, d, e, mu_maj, &c, &m, &mu);
    if (r == 2) { fate = ORC_FATE_CAP; break; }
    if (r == 1) { fate = ORC_FATE_ESCAPE; break; }
    if (fd && !pb->primary_only)
      fd_point(pb, seed, h, c.n_real, p, d, e, 1.0 - mu_photo(pb, m, e) / mu, 0, emit_w, ctx);
    if (draw(&s) * mu < mu_photo(pb, m, e)) { fate = ORC_FATE_ABSORBED; break; }
    double mu_c, eps;
    if (compton_sample(&s, e, &mu_c, &eps)) { fate = ORC_FATE_CAP; break; }
    double az = 2.0 * ORC_PI * draw(&s);
    orc_rotate(d, mu_c, az);
    e = eps * e;
    c.n_compton += 1;
    if (e < elow) { fate = ORC_FATE_BELOW_WINDOW; break; }
  }
  /* record the fate before detection so that the events land in rec */
  if (rec) {
    memset(rec, 0, sizeof(*rec));
    rec->fate = (uint8_t)fate;
  }
  /* Sec. 5.3 (dual-matrix OS): the back-projection matrix models attenuation
   * and detector blur only, i.e. photons that reach the camera unscattered */
  if (!pb->forced_detection && fate == ORC_FATE_ESCAPE && !(pb->primary_only && c.n_compton > 0))
    detect(pb, &s, p, d, emit, ctx);
  if (rec) {
    rec->n_virtual = c.n_virtual;
    rec->n_real = c.n_real;
    rec->n_compton = c.n_compton;
    rec->n_draws = s.n_draws;
    rec->e_final_kev = e;
  }
}

/* ------------------------------------------------------------------------ */
/* drivers                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_record *rec;
} rec_ctx;

static void emit_to_record(void *ctx, int32_t row) {
  orc_record *r = ((rec_ctx *)ctx)->rec;
  if (r->n_events < ORC_MAX_REC_EVENTS) r->event_row[r->n_events] = row;
  if (r->n_events < 255) r->n_events += 1;
}

/* Per-history trace records for histories first .. first+count-1. */
int orc_trace(const orc_problem *pb, uint64_t seed, uint64_t first, uint64_t count, orc_record *out) {
  double mu_maj = orc_majorant(pb);
  for (uint64_t i = 0; i < count; ++i) {
    rec_ctx ctx;
    ctx.rec = &out[i];
    memset(&out[i], 0, sizeof(out[i]));
    run_history(pb, seed, first + i, mu_maj, &out[i], emit_to_record, NULL, &ctx);
  }
  return 0;
}

/* Events of a history range, in history order (then view order). */
typedef struct {
  int32_t *row;
  int64_t *col;
  int64_t *q; /* fixed-point weights (1 for analog events) */
  int64_t n, cap;
  int64_t current_col;
  int64_t q_analog; /* weight of an analog detection: 1, or R8's rint(w 2^48) */
  int failed;
} ev_buf;

static void emit_to_buf_w(void *ctx, int32_t row, int64_t q) {
  ev_buf *b = (ev_buf *)ctx;
  if (b->failed) return;
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 1024;
    int32_t *nr = (int32_t *)realloc(b->row, (size_t)nc * sizeof(int32_t));
    if (!nr) { b->failed = 1; return; }
    b->row = nr;
    int64_t *ncl = (int64_t *)realloc(b->col, (size_t)nc * sizeof(int64_t));
    if (!ncl) { b->failed = 1; return; }
    b->col = ncl;
    int64_t *nq = (int64_t *)realloc(b->q, (size_t)nc * sizeof(int64_t));
    if (!nq) { b->failed = 1; return; }
    b->q = nq;
    b->cap = nc;
  }
  b->row[b->n] = row;
  b->col[b->n] = b->current_col;
  b->q[b->n] = q;
  b->n += 1;
}

static void emit_to_buf(void *ctx, int32_t row) { emit_to_buf_w(ctx, row, ((ev_buf *)ctx)->q_analog); }

typedef struct {
  const orc_problem *pb;
  uint64_t seed, first, count;
  double mu_maj;
  ev_buf buf;
  uint64_t fates[4];
} worker_arg;

static void *worker(void *arg) {
  worker_arg *w = (worker_arg *)arg;
  int64_t n_vox = (int64_t)w->pb->nx * w->pb->ny * w->pb->nz;
  w->buf.q_analog = w->pb->forced_direction ? (int64_t)llrint(orc_direction_band(w->pb) * ORC_FD_SCALE) : 1;
  for (uint64_t i = 0; i < w->count; ++i) {
    uint64_t h = w->first + i;
    orc_record rec;
    w->buf.current_col = (int64_t)(h % (uint64_t)n_vox);
    run_history(w->pb, w->seed, h, w->mu_maj, &rec, emit_to_buf, emit_to_buf_w, &w->buf);
    w->fates[rec.fate] += 1;
  }
  return NULL;
}

/* Run histories [first, first+count) on n_threads threads.  On success the
 * caller owns *rows/*cols (free with orc_free) holding *n_events events in
 * history order; fates[4] counts ABSORBED, BELOW_WINDOW, ESCAPE, CAP.
 * The result does not depend on n_threads. */
int orc_run_w(const orc_problem *pb, uint64_t seed, uint64_t first, uint64_t count, int n_threads, int32_t **rows,
              int64_t **cols, int64_t **qs, int64_t *n_events, uint64_t fates[4]) {
  if (n_threads < 1) n_threads = 1;
  if ((uint64_t)n_threads > count && count > 0) n_threads = (int)count;
  if (count == 0) n_threads = 1;
  double mu_maj = orc_majorant(pb);
  worker_arg *args = (worker_arg *)calloc((size_t)n_threads, sizeof(worker_arg));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!args || !th) { free(args); free(th); return -2; }
  uint64_t base = count / (uint64_t)n_threads, extra = count % (uint64_t)n_threads, start = first;
  for (int t = 0; t < n_threads; ++t) {
    uint64_t c = base + ((uint64_t)t < extra ? 1 : 0);
    args[t].pb = pb; args[t].seed = seed; args[t].first = start; args[t].count = c; args[t].mu_maj = mu_maj;
    start += c;
  }
  for (int t = 1; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &args[t]);
  worker(&args[0]);
  for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
  int64_t total = 0;
  int failed = 0;
  for (int t = 0; t < n_threads; ++t) { total += args[t].buf.n; failed |= args[t].buf.failed; }
  int32_t *r = NULL;
  int64_t *cl = NULL, *qq = NULL;
  if (!failed) {
    r = (int32_t *)malloc((size_t)(total ? total : 1) * sizeof(int32_t));
    cl = (int64_t *)malloc((size_t)(total ? total : 1) * sizeof(int64_t));
    qq = (int64_t *)malloc((size_t)(total ? total : 1) * sizeof(int64_t));
    if (!r || !cl || !qq) failed = 1;
  }
  int64_t off = 0;
  for (int t = 0; t < 4; ++t) fates[t] = 0;
  for (int t = 0; t < n_threads; ++t) {
    if (!failed && args[t].buf.n) {
      memcpy(r + off, args[t].buf.row, (size_t)args[t].buf.n * sizeof(int32_t));
      memcpy(cl + off, args[t].buf.col, (size_t)args[t].buf.n * sizeof(int64_t));
      memcpy(qq + off, args[t].buf.q, (size_t)args[t].buf.n * sizeof(int64_t));
      off += args[t].buf.n;
    }
    for (int f = 0; f < 4; ++f) fates[f] += args[t].fates[f];
    free(args[t].buf.row);
    free(args[t].buf.col);
    free(args[t].buf.q);
  }
  free(args);
  free(th);
  if (failed) { free(r); free(cl); free(qq); return -2; }
  *rows = r;
  *cols = cl;
  if (qs) *qs = qq; else free(qq);
  *n_events = total;
  return 0;
}

/* Analog events only (no weights): as orc_run_w without the weights. */
int orc_run(const orc_problem *pb, uint64_t seed, uint64_t first, uint64_t count, int n_threads, int32_t **rows,
            int64_t **cols, int64_t *n_events, uint64_t fates[4]) {
  return orc_run_w(pb, seed, first, count, n_threads, rows, cols, NULL, n_events, fates);
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* pins: pieces of the history exposed on their own                          */
/* ------------------------------------------------------------------------ */

/* Narrow beam: n photons of energy e start at p0 with direction d; photon i
 * uses the stream of history i.  Returns how many leave the box without a
 * real collision (the uncollided transmission count). */
uint64_t orc_beam(const orc_problem *pb, uint64_t seed, uint64_t n, const double p0[3], const double d[3],
                  double e_kev) {
  double mu_maj = orc_majorant(pb);
  uint64_t through = 0;
  for (uint64_t i = 0; i < n; ++i) {
    orc_stream s;
    stream_init(&s, seed, i);
    orc_counts c = {0, 0, 0, 0};
    double p[3] = {p0[0], p0[1], p0[2]};
    int m;
    double mu;
    if (woodcock_flight(pb, &s, p, d, e_kev, mu_maj, &c, &m, &mu) == 1) through += 1;
  }
  return through;
}

/* n Compton samples at energy e: cos(theta) and E'/E; sample i uses the
 * stream of history i.  Returns the number of samples that hit the cap. */
uint64_t orc_kn_sample(double e_kev, uint64_t seed, uint64_t n, double *cos_out, double *eps_out) {
  uint64_t capped = 0;
  for (uint64_t i = 0; i < n; ++i) {
    orc_stream s;
    stream_init(&s, seed, i);
    double mu = 0.0, eps = 0.0;
    if (compton_sample(&s, e_kev, &mu, &eps)) capped += 1;
    cos_out[i] = mu;
    eps_out[i] = eps;
  }
  return capped;
}

/* The first n uniforms of history h's stream (as doubles in (0,1)). */
void orc_uniforms(uint64_t seed, uint64_t h, uint64_t n, double *out) {
  orc_stream s;
  stream_init(&s, seed, h);
  for (uint64_t i = 0; i < n; ++i) out[i] = draw(&s);
}

/* Detection only: offer a photon at p with direction d to the views, using
 * the stream of history h; writes up to max_rows rows and returns how many
 * detections there were. */
typedef struct {
  int32_t *rows;
  int max_rows, n;
} det_ctx;

static void emit_to_det(void *ctx, int32_t row) {
  det_ctx *c = (det_ctx *)ctx;
  if (c->n < c->max_rows) c->rows[c->n] = row;
  c->n += 1;
}

int orc_detect(const orc_problem *pb, uint64_t seed, uint64_t h, const double p[3], const double d[3],
               int32_t *rows, int max_rows) {
  orc_stream s;
  stream_init(&s, seed, h);
  det_ctx ctx = {rows, max_rows, 0};
  detect(pb, &s, p, d, emit_to_det, &ctx);
  return ctx.n;
}

/* Forced copies of one interaction (R7), for the pins: writes up to
 * max_rows (row, q) pairs and returns how many there were. */
typedef struct {
  int32_t *rows;
  int64_t *qs;
  int max_rows, n;
} fdp_ctx;

static void emit_to_fdp(void *ctx, int32_t row, int64_t q) {
  fdp_ctx *c = (fdp_ctx *)ctx;
  if (c->n < c->max_rows) { c->rows[c->n] = row; c->qs[c->n] = q; }
  c->n += 1;
}

int orc_fd_point(const orc_problem *pb, uint64_t seed, uint64_t h, uint32_t n, const double p[3], const double d_in[3],
                 double e_kev, double p_keep, int emission, int32_t *rows, int64_t *qs, int max_rows) {
  fdp_ctx ctx = {rows, qs, max_rows, 0};
  fd_point(pb, seed, h, n, p, d_in, e_kev, p_keep, emission, emit_to_fdp, &ctx);
  return ctx.n;
}
