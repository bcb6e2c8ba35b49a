"""Pins for the oracle's transport physics against closed forms.

Each test fixes one part of the history (paper Sec. 2: sampling from the
cross-sections; Sec. 3: scatter lowers the energy and turns the photon,
parallel-hole collimation, the energy window) with a result that does not
come from the oracle's own code: the Klein-Nishina formula integrated by
quadrature, Beer-Lambert transmission, the collimator's acceptance
integral, the Gaussian CDF and the symmetry of the set-up.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle
from paper_2105_13324_gb300 import phantoms as P

RE = 2.8179403262e-13
MEC2 = 510.99895


def kn_dsigma_domega(mu, e_kev):
    """Klein-Nishina differential cross-section per electron (cm^2/sr)."""
    a = e_kev / MEC2
    eps = 1.0 / (1.0 + a * (1.0 - mu))
    return 0.5 * RE * RE * eps * eps * (eps + 1.0 / eps - (1.0 - mu * mu))


@pytest.mark.parametrize("e_kev", [20.0, 71.0, 126.45, 140.5, 167.0, 511.0])
def test_sigma_kn_equals_integral_of_differential(e_kev):
    want, _ = integrate.quad(lambda mu: 2.0 * math.pi * kn_dsigma_domega(mu, e_kev), -1.0, 1.0,
                             epsabs=0, epsrel=1e-13)
    assert oracle.sigma_kn_cm2(e_kev) == pytest.approx(want, rel=1e-11)


def test_sigma_kn_thomson_limit_and_value_at_tc99m():
    thomson = 8.0 * math.pi / 3.0 * RE * RE
    assert oracle.sigma_kn_cm2(0.01) == pytest.approx(thomson, rel=1e-4)
    assert oracle.sigma_kn_cm2(140.5) * 1e24 == pytest.approx(0.451849, abs=2e-6)


def test_attenuation_of_water_and_majorant():
    w = P.workload("water32")
    pr = oracle.Problem(w.phantom, w.geometry)
    # stated attenuation of water at 140.5 keV: 0.154 /cm = 0.0154 /mm
    assert oracle.mu_total(pr, 1, 140.5) == pytest.approx(0.0154, rel=1e-5)
    es = np.linspace(126.45, 140.5, 30)
    mus = [oracle.mu_total(pr, 1, e) for e in es]
    assert all(a > b for a, b in zip(mus, mus[1:]))           # falls with energy
    assert oracle.majorant(pr) == max(oracle.mu_total(pr, m, 126.45) for m in range(2))
    # air: same physics at 1/830 of the density
    assert oracle.mu_total(pr, 0, 140.5) < 2e-3 * oracle.mu_total(pr, 1, 140.5)


def test_compton_polar_angle_matches_klein_nishina():
    e = 140.5
    cos_t, eps, capped = oracle.kn_sample(e, seed=11, n=400_000)
    assert capped == 0
    edges = np.linspace(-1.0, 1.0, 41)
    obs, _ = np.histogram(cos_t, edges)
    tot, _ = integrate.quad(lambda m: kn_dsigma_domega(m, e), -1, 1)
    exp = np.array([integrate.quad(lambda m: kn_dsigma_domega(m, e), a, b)[0] / tot
                    for a, b in zip(edges[:-1], edges[1:])]) * len(cos_t)
    chi2 = np.sum((obs - exp) ** 2 / exp)
    assert stats.chi2.sf(chi2, len(obs) - 1) > 0.01
    # scattered energy follows the Compton relation E'/E = 1/(1 + a(1 - cos))
    a = e / MEC2
    np.testing.assert_allclose(eps, 1.0 / (1.0 + a * (1.0 - cos_t)), rtol=1e-15)


def test_fraction_of_scatters_staying_in_window():
    e, elow = 140.5, 126.45
    a = e / MEC2
    mu_min = 1.0 - (e / elow - 1.0) / a          # E' >= elow  <=>  cos >= mu_min
    tot, _ = integrate.quad(lambda m: kn_dsigma_domega(m, e), -1, 1)
    part, _ = integrate.quad(lambda m: kn_dsigma_domega(m, e), mu_min, 1)
    frac = part / tot
    assert frac == pytest.approx(0.33439, abs=5e-5)
    _, eps, _ = oracle.kn_sample(e, seed=12, n=300_000)
    got = np.mean(eps * e >= elow)
    assert abs(got - frac) < 4.0 * math.sqrt(frac * (1 - frac) / len(eps))


@pytest.mark.parametrize("d", [(0.3, -0.5, 0.812404), (0.0, 0.0, 1.0), (0.0, 0.0, -1.0), (1.0, 0.0, 0.0)])
def test_rotation_turns_by_the_polar_angle(d):
    d = np.asarray(d) / np.linalg.norm(d)
    rng = np.random.default_rng(3)
    outs = []
    for mu, phi in zip(rng.uniform(-1, 1, 200), rng.uniform(0, 2 * np.pi, 200)):
        n = oracle.rotate(d, mu, phi)
        assert np.linalg.norm(n) == pytest.approx(1.0, abs=1e-14)
        assert float(n @ d) == pytest.approx(mu, abs=1e-9)
        outs.append(n)
    # azimuths about d are spread over the whole circle
    outs = np.asarray(outs)
    perp = outs - np.outer(outs @ d, d)
    assert np.linalg.norm(perp.mean(axis=0)) < 0.2


def _beam_fraction(row, thickness_mm, extra_rows=(), n=200_000, seed=5):
    n_vox, h = 40, 4.0
    ph = P.slab_phantom(n_vox, h, row, thickness_mm, extra_rows)
    g = P.spect_geometry(1, 180.0, 8, 4.0, n_vox, h)
    pr = oracle.Problem(ph, g)
    p0 = (-0.5 * n_vox * h + 1e-9, 0.5, 0.5)
    through = oracle.beam(pr, seed, n, p0, (1.0, 0.0, 0.0), 140.5)
    mu = oracle.mu_total(pr, 1, 140.5)
    path = float(np.count_nonzero(ph.material[0, 0, :] == 1)) * h   # slab voxels on the beam line
    return through / n, math.exp(-mu * path), n


@pytest.mark.parametrize("row,thick,extra", [
    (P.WATER, 96.0, ()),
    (P.BONE, 48.0, ()),
    (P.WATER, 96.0, (P.BONE,)),     # majorant far above mu: virtual collisions are unbiased
])
def test_narrow_beam_transmission_is_beer_lambert(row, thick, extra):
    got, want, n = _beam_fraction(row, thick, extra)
    sd = math.sqrt(want * (1 - want) / n)
    assert abs(got - want) < 4.0 * sd


def _problem(n_vox, h, views, arc, bins, bin_mm, phantom=None, **kw):
    ph = phantom if phantom is not None else P.vacuum_phantom(n_vox, h)
    g = P.Geometry(n_views=views, arc_deg=arc, n_bins_u=bins, n_bins_v=bins, bin_mm=bin_mm,
                   radius_mm=P.front_face_radius(n_vox, h), **kw)
    return ph, g, oracle.Problem(ph, g)


def test_collimator_acceptance_integral():
    # unattenuated isotropic source: per-view detection probability
    #   P = 1/2 int_0^1 f(x) t / (1 + t^2)^(3/2) dt/dx dx,  t = x d/L,
    # f(x) = (2/pi)(acos x - x sqrt(1-x^2)); small-angle limit (1/16)(d/L)^2.
    L, d = 5.0, 1.5
    ph, g, pr = _problem(4, 1.0, 8, 360.0, 64, 4.0, hole_len_mm=L, hole_diam_mm=d, fwhm_mm=0.5)

    def integrand(x):
        t = x * d / L
        f = (2 / math.pi) * (math.acos(x) - x * math.sqrt(1 - x * x))
        return 0.5 * f * t / (1 + t * t) ** 1.5 * (d / L)

    p_view, _ = integrate.quad(integrand, 0, 1, epsabs=0, epsrel=1e-12)
    assert integrate.quad(lambda x: (2 / math.pi) * (math.acos(x) - x * math.sqrt(1 - x * x)) * x, 0, 1)[0] \
        == pytest.approx(1 / 8, rel=1e-10)
    assert p_view == pytest.approx((d / L) ** 2 / 16, rel=0.1)
    H = 400_000
    rows, cols, fates = oracle.run(pr, 9, 0, H, threads=4)
    assert fates[oracle.FATE_ESCAPE] == H
    per_view = np.bincount(rows // (64 * 64), minlength=8)
    want = p_view * H
    assert np.all(np.abs(per_view - want) < 4.0 * math.sqrt(want))


def test_blur_profile_is_gaussian_and_bins_are_placed():
    fwhm, binw, B = 3.5, 0.25, 128
    ph, g, pr = _problem(4, 1.0, 4, 360.0, B, binw, fwhm_mm=fwhm)
    sigma = fwhm / (2 * math.sqrt(2 * math.log(2)))
    # photon on the axis of view 0, moving along its normal: always accepted
    iu = []
    for h in range(20_000):
        rows, n = oracle.detect(pr, 3, h, (0.0, 0.0, 0.0), (1.0, 0.0, 0.0))
        assert n <= 1
        if n:
            assert rows[0] // (B * B) == 0
            iu.append(rows[0] % B)
    iu = np.asarray(iu)
    assert len(iu) > 19_900        # a few land beyond +-16 mm only
    edges = (np.arange(B + 1) - B / 2) * binw
    p = np.diff(special.ndtr(edges / sigma))
    obs = np.bincount(iu, minlength=B)
    keep = p * len(iu) > 5
    exp = p[keep] * len(iu)
    chi2 = np.sum((obs[keep] - exp) ** 2 / exp)
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-3


def test_detector_axes_and_row_layout():
    B, binw = 64, 1.0
    ph, g, pr = _problem(4, 1.0, 4, 360.0, B, binw, fwhm_mm=1e-9)
    cases = [
        # (point, direction, view, transaxial offset a, axial offset b)
        ((0.0, 10.3, -5.7), (1.0, 0.0, 0.0), 0, 10.3, -5.7),
        ((10.3, 0.0, 2.2), (0.0, 1.0, 0.0), 1, -10.3, 2.2),   # view 90 deg: t = (-1, 0, 0)
        ((0.0, -7.6, 3.1), (-1.0, 0.0, 0.0), 2, 7.6, 3.1),    # view 180 deg: t = (0, -1, 0)
    ]
    for p, d, k, a, b in cases:
        rows, n = oracle.detect(pr, 1, 0, p, d)
        assert n == 1
        iu, iv = math.floor(a / binw + B / 2), math.floor(b / binw + B / 2)
        assert rows[0] == (k * B + iv) * B + iu


def test_fates_conserve_histories_and_threads_do_not_matter():
    w = P.workload("water32")
    pr = oracle.Problem(w.phantom, w.geometry)
    H = 300_000
    r1, c1, f1 = oracle.run(pr, 1, 0, H, threads=1)
    r3, c3, f3 = oracle.run(pr, 1, 0, H, threads=3)
    assert int(f1.sum()) == H and f1[oracle.FATE_CAP] == 0
    np.testing.assert_array_equal(r1, r3)
    np.testing.assert_array_equal(c1, c3)
    np.testing.assert_array_equal(f1, f3)
    # a history id range splits exactly: [0, H) = [0, m) ++ [m, H)
    m = 123_457
    ra, ca, fa = oracle.run(pr, 1, 0, m, threads=2)
    rb, cb, fb = oracle.run(pr, 1, m, H - m, threads=2)
    np.testing.assert_array_equal(np.concatenate([ra, rb]), r1)
    np.testing.assert_array_equal(np.concatenate([ca, cb]), c1)
    np.testing.assert_array_equal(fa + fb, f1)
    # each event's column is the voxel its history started in
    rec = oracle.trace(pr, 1, 0, 50_000)
    assert np.all(rec["n_events"][rec["fate"] != oracle.FATE_ESCAPE] == 0)
    assert np.all(rec["e_final_kev"][rec["fate"] == oracle.FATE_ESCAPE] >= 126.45)
    assert np.all(rec["e_final_kev"][rec["fate"] == oracle.FATE_BELOW_WINDOW] < 126.45)
    assert np.all(rec["n_compton"][rec["fate"] == oracle.FATE_BELOW_WINDOW] >= 1)


def test_views_of_a_symmetric_setup_see_equal_counts():
    # centred water cylinder on a cubic grid, views 90 deg apart: the set-up
    # is invariant under the 90-degree rotation, so per-view totals agree
    ph = P.water_cylinder_phantom(n=16, h=4.0, radius=28.0)
    g = P.Geometry(n_views=4, arc_deg=360.0, n_bins_u=24, n_bins_v=24, bin_mm=4.0,
                   radius_mm=P.front_face_radius(16, 4.0), hole_len_mm=10.0, hole_diam_mm=2.0)
    pr = oracle.Problem(ph, g)
    rows, cols, fates = oracle.run(pr, 4, 0, 2_000_000, threads=8)
    per_view = np.bincount(rows // (24 * 24), minlength=4)
    chi2 = np.sum((per_view - per_view.mean()) ** 2 / per_view.mean())
    assert stats.chi2.sf(chi2, 3) > 1e-3
    # and attenuation matters: the count is below the vacuum acceptance
    assert per_view.sum() > 100


def test_histories_per_voxel_by_brute_force():
    for n_vox, first, count in [(7, 0, 50), (7, 3, 0), (13, 11, 100), (5, 1000, 17)]:
        want = np.bincount(np.arange(first, first + count) % n_vox, minlength=n_vox)
        np.testing.assert_array_equal(oracle.histories_per_voxel(n_vox, first, count), want)


def test_system_counts_by_brute_force():
    rng = np.random.default_rng(0)
    rows = rng.integers(0, 9, 500).astype(np.int32)
    cols = rng.integers(0, 6, 500)
    c = oracle.system_counts(rows, cols, 9, 6).toarray()
    want = np.zeros((9, 6), np.int64)
    for r, q in zip(rows, cols):
        want[r, q] += 1
    np.testing.assert_array_equal(c, want)


def test_unscattered_photons_keep_the_source_energy_and_scattered_ones_obey_compton():
    # traces: an escape without scattering leaves at exactly E0 = 140.5 keV;
    # after one scatter the energy lies in [E0 / (1 + 2 E0 / m c^2), E0)
    w = P.workload("water32")
    rec = oracle.trace(oracle.Problem(w.phantom, w.geometry), w.seed, 0, 200_000)
    esc = rec["fate"] == oracle.FATE_ESCAPE
    prim = esc & (rec["n_compton"] == 0)
    assert prim.sum() > 10_000
    assert np.all(rec["e_final_kev"][prim] == 140.5)
    one = esc & (rec["n_compton"] == 1)
    e1 = rec["e_final_kev"][one]
    assert one.sum() > 1000
    assert np.all(e1 < 140.5) and np.all(e1 >= 140.5 / (1 + 2 * 140.5 / MEC2) * (1 - 1e-12))
    assert np.all(e1 >= (1 - 0.5 * w.geometry.window_frac) * 140.5)   # still in the window


def test_emission_is_uniform_in_its_voxel_and_detected_at_its_axial_position():
    # vacuum, 2^3 voxels of 16 mm, a narrow collimator (d/L = 0.03, crystal
    # ~70 mm from the source: axial spread ~1 mm), 1 mm bins, almost no blur.
    # The axial bin of a detection is then the emission height up to that
    # spread, so relative to its voxel's centre the detections are centred
    # (by symmetry, whatever the spread), lie within the voxel's 16 mm (plus
    # the spread), and are flat away from the voxel's faces.
    n, h = 2, 16.0
    ph = P.vacuum_phantom(n, h)
    g = P.Geometry(n_views=4, arc_deg=360.0, n_bins_u=80, n_bins_v=80, bin_mm=1.0,
                   radius_mm=P.front_face_radius(n, h), hole_len_mm=20.0, hole_diam_mm=0.6, fwhm_mm=0.01)
    pr = oracle.Problem(ph, g)
    rows, cols, _ = oracle.run(pr, 3, 0, 20_000_000, threads=4)
    iv = (rows // 80) % 80
    z = (iv + 0.5) - 40.0                            # bin centre, mm (grid centred on 0)
    zc = (cols // (n * n)) * h - 0.5 * n * h + 0.5 * h  # centre height of the emitting voxel
    rel = z - zc
    assert len(rel) > 3000
    assert np.all(np.abs(rel) <= 0.5 * h + 2.5)
    assert abs(rel.mean()) < 4 * (h / math.sqrt(12)) / math.sqrt(len(rel))
    counts = np.histogram(rel, bins=12, range=(-6.0, 6.0))[0]   # central 12 mm: flat
    exp = counts.sum() / 12
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < stats.chi2.ppf(0.9999, 11)
