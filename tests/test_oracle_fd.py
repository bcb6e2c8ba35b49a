"""Pins for the oracle's forced detection (the variance-reduction section of
the paper: a weighted copy of the photon is forced to the detector at each
interaction location).

Forced detection is an unbiased estimator of the same detection
probabilities the analog transport estimates, so the strongest pin is the
analog oracle itself, run with many more histories: per view and per block
of detector bins the two agree within their statistical errors, for the
full matrix and for the unscattered (primary) part.  Its pieces are pinned
on their own against closed forms: the transmission along a ray against
Beer-Lambert with analytic chord lengths, the Klein-Nishina angular density
against its normalisation and forward value, and, in vacuum, the forced
weight against the collimator's acceptance integral.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2105_13324_gb300 import phantoms as P

RE = 2.8179403262e-13


def _ray_box_exit(p, d, half):
    t = np.inf
    for a in range(3):
        if d[a] > 0:
            t = min(t, (half[a] - p[a]) / d[a])
        elif d[a] < 0:
            t = min(t, (-half[a] - p[a]) / d[a])
    return t


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def test_transmission_uniform_grid_is_beer_lambert():
    ph = P.uniform_phantom(8, 5.0)
    g = P.spect_geometry(4, 360.0, 8, 5.0, 8, 5.0)
    pr = oracle.Problem(ph, g)
    rng = np.random.default_rng(3)
    half = np.array([20.0, 20.0, 20.0])
    for e in (140.5, 126.45, 90.0):
        mu = oracle.mu_total(pr, 1, e)
        for _ in range(200):
            p = rng.uniform(-19.9, 19.9, 3)
            d = _unit(rng)
            want = math.exp(-mu * _ray_box_exit(p, d, half))
            assert oracle.transmission(pr, p, d, e) == pytest.approx(want, rel=1e-12)
    # axis-aligned rays (two direction components exactly 0)
    for a in range(3):
        for sgn in (1.0, -1.0):
            d = np.zeros(3)
            d[a] = sgn
            p = np.array([1.3, -2.7, 4.1])
            mu = oracle.mu_total(pr, 1, 140.5)
            want = math.exp(-mu * _ray_box_exit(p, d, half))
            assert oracle.transmission(pr, p, d, 140.5) == pytest.approx(want, rel=1e-12)


def test_transmission_without_a_direction_is_undefined():
    # a zero or NaN direction never leaves the grid: NaN, not an endless walk
    ph = P.uniform_phantom(8, 5.0)
    g = P.spect_geometry(4, 360.0, 8, 5.0, 8, 5.0)
    pr = oracle.Problem(ph, g)
    for d in (np.zeros(3), np.full(3, np.nan)):
        assert math.isnan(oracle.transmission(pr, np.array([1.0, 2.0, 3.0]), d, 140.5))


def test_transmission_through_layers_by_chord_lengths():
    # z-layers of water and bone over vacuum: the exponent is the sum over
    # layers of mu times the length of the ray inside the layer
    n, h = 10, 4.0
    ph = P.vacuum_phantom(n, h)
    ph.rho, ph.z_over_a, ph.z_eff = (np.array([0.0, 1.0, 1.85]), np.array([0.5, 0.55509, 0.5148]),
                                     np.array([7.0, 7.42, 13.0]))
    layer_mat = np.array([0, 1, 1, 2, 0, 1, 2, 2, 1, 0], np.uint8)
    ph.material = np.ascontiguousarray(np.broadcast_to(layer_mat[:, None, None], (n, n, n)))
    pr = oracle.Problem(ph, P.spect_geometry(4, 360.0, 8, 4.0, n, h))
    rng = np.random.default_rng(5)
    half = np.full(3, n * h / 2)
    mus = [oracle.mu_total(pr, m, 140.5) for m in range(3)]
    for _ in range(300):
        p = rng.uniform(-19.5, 19.5, 3)
        d = _unit(rng)
        t_exit = _ray_box_exit(p, d, half)
        expo = 0.0
        for k in range(n):
            z0, z1 = -half[2] + k * h, -half[2] + (k + 1) * h
            if d[2] != 0:
                ta, tb = sorted(((z0 - p[2]) / d[2], (z1 - p[2]) / d[2]))
            else:
                ta, tb = (-np.inf, np.inf) if z0 <= p[2] < z1 else (0.0, 0.0)
            lo, hi = max(ta, 0.0), min(tb, t_exit)
            if hi > lo:
                expo += mus[layer_mat[k]] * (hi - lo)
        assert oracle.transmission(pr, p, d, 140.5) == pytest.approx(math.exp(-expo), rel=1e-11)


@pytest.mark.parametrize("e_kev", [30.0, 90.0, 140.5, 364.0])
def test_kn_angular_density_is_normalised(e_kev):
    total, _ = integrate.quad(lambda mu: 2 * math.pi * oracle.kn_pdf_sr(e_kev, mu), -1, 1, epsabs=0,
                              epsrel=1e-12)
    assert total == pytest.approx(1.0, rel=1e-10)
    # forward scattering: dsigma/dOmega(0) = r_e^2 (eps = 1)
    assert oracle.kn_pdf_sr(e_kev, 1.0) == pytest.approx(RE * RE / oracle.sigma_kn_cm2(e_kev), rel=1e-13)


def test_forced_weight_in_vacuum_is_the_acceptance_integral():
    # one emission point at the centre of a vacuum grid: the mean forced
    # weight per view is (1 / 4 pi) int_cone f dOmega, the per-view
    # detection probability of an isotropic source
    L, dh = 20.0, 2.0
    ph = P.vacuum_phantom(4, 2.0)
    g = P.Geometry(n_views=6, arc_deg=360.0, n_bins_u=64, n_bins_v=64, bin_mm=2.0,
                   radius_mm=P.front_face_radius(4, 2.0), hole_len_mm=L, hole_diam_mm=dh, fwhm_mm=1.0)
    pr = oracle.Problem(ph, g, forced_detection=True)

    def integrand(th):
        x = (L / dh) * math.tan(th)
        return 2 * math.pi * (2 / math.pi) * (math.acos(x) - x * math.sqrt(1 - x * x)) * math.sin(th)

    want = integrate.quad(integrand, 0, math.atan(dh / L), epsabs=0, epsrel=1e-12)[0] / (4 * math.pi)
    ws = []
    for h in range(4000):
        rows, q = oracle.fd_point(pr, 7, h, 0, [0.1, -0.2, 0.3], [0, 0, 1], 140.5, 1.0, True)
        assert len(rows) == 6                       # every view gets a copy (nothing attenuates)
        assert np.all(rows // (64 * 64) == np.arange(6))
        ws.append(q / oracle.FD_SCALE)
    ws = np.array(ws)
    m, se = ws.mean(), ws.std() / math.sqrt(ws.size)
    assert abs(m - want) < 4 * se
    assert se < 0.01 * want
    # the copy lands near the projection of the point: the centre bins +- blur
    assert np.all(np.abs(rows % 64 - 32) <= 3) and np.all(np.abs((rows // 64) % 64 - 32) <= 3)


def test_forced_collision_weight_is_the_scatter_integral():
    # one collision at the centre of a uniform water grid, incoming direction
    # at 60 degrees to view 0's normal: the mean forced weight of view 0 is
    #   p_keep int_cone p_KN(d_in . d | E) f(x) exp(-mu(E'(d)) t_exit(d)) dOmega
    # (E' from the Compton relation), by quadrature over the cone
    L, dh, n, h = 20.0, 2.0, 10, 6.0
    ph = P.uniform_phantom(n, h)
    g = P.Geometry(n_views=1, arc_deg=360.0, n_bins_u=64, n_bins_v=64, bin_mm=4.0,
                   radius_mm=P.front_face_radius(n, h), hole_len_mm=L, hole_diam_mm=dh, fwhm_mm=1.0,
                   window_frac=0.5)
    pr = oracle.Problem(ph, g, forced_detection=True)
    e, p_keep = 140.5, 0.83
    p0 = np.array([1.0, -2.0, 0.5])
    d_in = np.array([math.cos(math.radians(60)), math.sin(math.radians(60)), 0.0])
    half = np.full(3, n * h / 2)
    tmax = math.atan(dh / L)

    def integrand(ph_, th):
        d = np.array([math.cos(th), math.sin(th) * math.cos(ph_), math.sin(th) * math.sin(ph_)])
        mu_s = float(d_in @ d)
        e1 = e / (1 + e / 510.99895 * (1 - mu_s))
        x = (L / dh) * math.tan(th)
        f = (2 / math.pi) * (math.acos(x) - x * math.sqrt(1 - x * x))
        mu = oracle.mu_total(pr, 1, e1)
        return oracle.kn_pdf_sr(e, mu_s) * f * math.exp(-mu * _ray_box_exit(p0, d, half)) * math.sin(th)

    want = p_keep * integrate.dblquad(integrand, 0, tmax, 0, 2 * math.pi, epsabs=0, epsrel=1e-9)[0]
    ws = np.zeros(60000)
    for hh in range(ws.size):
        rows, q = oracle.fd_point(pr, 11, hh, 2, p0, d_in, e, p_keep, False)
        ws[hh] = q.sum() / oracle.FD_SCALE
    m, se = ws.mean(), ws.std() / math.sqrt(ws.size)
    assert se < 0.005 * want
    assert abs(m - want) < 4 * se


def _small_problem(forced: bool, primary: bool = False, medium: str = "water+bone"):
    # 16^3 x 4 mm; a wide window (E >= 0.75 E0) so that scatter is a sizeable
    # part of the counts.  "water+bone": water cylinder with a bone core
    # (photo-absorption ~17 % of bone's attenuation at 140 keV);
    # "high-z": a cylinder of Z_eff 20 (photo-absorption ~55 %), where the
    # survival factor of the collision copies matters most
    ph = P.water_cylinder_phantom(16, 4.0, radius=24.0, shell_outer=(14.0, 12.0, 12.0), wall=5.0)
    c = P.voxel_centres(16, 4.0)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    ph.material = ph.material.copy()
    if medium == "water+bone":
        core = (xx - 6.0) ** 2 + yy ** 2 <= 10.0 ** 2
        ph.material[:, core] = 2
        extra = (1.85, 0.5148, 13.0)
    else:
        ph.material[ph.material == 1] = 2
        extra = (1.0, 0.5, 20.0)
    ph.rho, ph.z_over_a, ph.z_eff = (np.append(ph.rho, extra[0]), np.append(ph.z_over_a, extra[1]),
                                     np.append(ph.z_eff, extra[2]))
    g = P.spect_geometry(8, 360.0, 16, 4.0, 16, 4.0, hole_len_mm=20.0, hole_diam_mm=2.0, fwhm_mm=4.0,
                         window_frac=0.5)
    return ph, g, oracle.Problem(ph, g, primary_only=primary, forced_detection=forced)


def _blocks(rows, w):
    # view x (4 x 4 blocks of bins): 8 * 16 aggregates
    k = rows // 256
    iv = (rows // 16) % 16
    iu = rows % 16
    b = (k * 4 + iv // 4) * 4 + iu // 4
    return np.bincount(b, weights=w, minlength=8 * 16)


def _moments(rows, w):
    # per view: weight, and first moments of the transaxial and axial bin
    k = rows // 256
    iv = (rows // 16) % 16
    iu = rows % 16
    ww = np.ones(len(rows)) if w is None else w
    return np.stack([np.bincount(k, weights=ww * t, minlength=8) for t in (np.ones(len(rows)), iu, iv)])


def _z(fd_batches, analog_sum, analog_sumsq, H_a):
    # fd_batches: per-batch estimates (per history); analog: sums of x and
    # x^2 over H_a histories (events are 0/1 per view and history)
    n_b = fd_batches.shape[0]
    fd = fd_batches.mean(axis=0)
    var_f = fd_batches.var(axis=0, ddof=1) / n_b
    an = analog_sum / H_a
    var_a = analog_sumsq / H_a ** 2
    return (fd - an) / np.sqrt(var_a + var_f)


N_SMALL = 16 ** 3


def _analog_and_fd(medium, primary, h_a=1024 * N_SMALL, n_batch=16):
    _, _, pa = _small_problem(False, primary, medium)
    _, _, pf = _small_problem(True, primary, medium)
    ra, ca, _ = oracle.run(pa, 21, 0, h_a)
    fd = []
    for b in range(n_batch):                                  # each batch covers every voxel once
        rf, cf, q, _ = oracle.run_fd(pf, 33, b * N_SMALL, N_SMALL)
        fd.append((rf, q / oracle.FD_SCALE))
    return (ra, ca), fd


@pytest.mark.parametrize("medium,primary", [("water+bone", False), ("water+bone", True), ("high-z", False)])
def test_forced_detection_agrees_with_analog_transport(medium, primary):
    H_a = 1024 * N_SMALL
    (ra, _), fd = _analog_and_fd(medium, primary, H_a)
    # blocks of bins
    blk = np.array([_blocks(r, w) for r, w in fd]) / N_SMALL
    ab = _blocks(ra, None)
    z = _z(blk, ab, ab, H_a)
    assert np.all(np.isfinite(z))
    assert np.max(np.abs(z)) < 5.0
    assert np.mean(z * z) < 1.6
    # per view: total and the first moments of the bin position (the
    # moments' analog variance from the sum of squares of the bin indices)
    mom = np.array([_moments(r, w) for r, w in fd]) / N_SMALL
    am = _moments(ra, None)
    k = ra // 256
    sq = np.stack([np.bincount(k, weights=t * t, minlength=8).astype(np.float64)
                   for t in (np.ones(len(ra)), ra % 16, (ra // 16) % 16)])
    zm = _z(mom, am, sq, H_a)
    assert np.max(np.abs(zm)) < 4.5


def test_forced_detection_scatter_part_agrees_with_analog():
    # scatter = all - primary, history by history (same seeds): analog events
    # of scattered photons against the forced copies made at collisions
    H_a = 2048 * N_SMALL
    for medium in ("water+bone", "high-z"):
        (ra, _), fd_all = _analog_and_fd(medium, False, H_a)
        (rp, _), fd_pri = _analog_and_fd(medium, True, H_a)
        sa = np.bincount(ra // 256, minlength=8) - np.bincount(rp // 256, minlength=8)
        assert np.all(sa > 150)
        sf = np.array([np.bincount(r1 // 256, weights=w1, minlength=8) - np.bincount(r2 // 256, weights=w2, minlength=8)
                       for (r1, w1), (r2, w2) in zip(fd_all, fd_pri)]) / N_SMALL
        z = _z(sf.sum(axis=1, keepdims=True), np.array([sa.sum()]), np.array([sa.sum()]), H_a)
        assert abs(z[0]) < 4.0
        zv = _z(sf, sa, sa, H_a)
        assert np.max(np.abs(zv)) < 4.5


def test_forced_primary_is_the_emission_part_and_threads_do_not_matter():
    _, _, pf = _small_problem(True, False)
    _, _, pp = _small_problem(True, True)
    rf, cf, qf, ff = oracle.run_fd(pf, 5, 100, 3000, threads=1)
    rf4, cf4, qf4, ff4 = oracle.run_fd(pf, 5, 100, 3000, threads=4)
    assert np.array_equal(rf, rf4) and np.array_equal(cf, cf4) and np.array_equal(qf, qf4)
    assert np.array_equal(ff, ff4)
    rp, cp, qp, _ = oracle.run_fd(pp, 5, 100, 3000, threads=3)
    # the primary events are a sub-multiset of the full ones (the emission copies)
    full = set(zip(cf.tolist(), rf.tolist(), qf.tolist()))
    assert all(t in full for t in zip(cp.tolist(), rp.tolist(), qp.tolist()))
    assert 0 < len(rp) < len(rf)
    assert qp.sum() < qf.sum()


def test_weighted_tally_sums_are_exact_integers():
    rng = np.random.default_rng(8)
    rows = rng.integers(0, 50, 5000).astype(np.int32)
    cols = rng.integers(0, 40, 5000).astype(np.int64)
    q = rng.integers(1, 2 ** 40, 5000).astype(np.int64)
    w = oracle.system_weights(rows, cols, q, 50, 40)
    dense = np.zeros((50, 40), np.int64)
    np.add.at(dense, (rows, cols), q)
    assert np.array_equal(w.toarray() * oracle.FD_SCALE, dense.astype(np.float64))
    assert w.nnz == np.count_nonzero(dense)


def test_forced_direction_in_vacuum_is_the_acceptance_integral():
    # vacuum, isotropic emission: with the band |cos theta| < sin(psi_max)
    # and weight sin(psi_max) per detection, the mean weight per history and
    # view is the per-view detection probability (1/4 pi) int_cone f dOmega
    L, dh = 20.0, 2.0
    ph = P.vacuum_phantom(4, 2.0)
    g = P.Geometry(n_views=6, arc_deg=360.0, n_bins_u=64, n_bins_v=64, bin_mm=2.0,
                   radius_mm=P.front_face_radius(4, 2.0), hole_len_mm=L, hole_diam_mm=dh, fwhm_mm=1.0)
    pr = oracle.Problem(ph, g, primary_only=True, forced_direction=True)
    band = oracle.direction_band(pr)
    assert band == pytest.approx(math.sin(math.atan(dh / L)), rel=1e-15)

    def integrand(th):
        x = (L / dh) * math.tan(th)
        return 2 * math.pi * (2 / math.pi) * (math.acos(x) - x * math.sqrt(1 - x * x)) * math.sin(th)

    want = integrate.quad(integrand, 0, math.atan(dh / L), epsabs=0, epsrel=1e-12)[0] / (4 * math.pi)
    H = 200_000
    rows, cols, q, fates = oracle.run_fd(pr, 4, 0, H, threads=4)
    assert np.all(q == round(band * oracle.FD_SCALE))
    per_view = np.bincount(rows // (64 * 64), minlength=6)
    # counts per view are binomial with p = want / band; weights w = band
    p = want / band
    assert np.all(np.abs(per_view - p * H) < 4.5 * math.sqrt(H * p * (1 - p)))
    with pytest.raises(ValueError):
        oracle.Problem(ph, g, forced_direction=True)


def test_forced_direction_primary_agrees_with_analog_primary():
    _, _, pa = _small_problem(False, True)
    ph, g, _ = _small_problem(False, True)
    pf = oracle.Problem(ph, g, primary_only=True, forced_direction=True)
    N = N_SMALL
    H_a = 1024 * N
    ra, _, _ = oracle.run(pa, 21, 0, H_a)
    blk = []
    for b in range(16):
        rf, _, q, _ = oracle.run_fd(pf, 41, b * 16 * N, 16 * N)
        blk.append(_blocks(rf, q / oracle.FD_SCALE) / (16 * N))
    blk = np.array(blk)
    ab = _blocks(ra, None)
    z = _z(blk, ab, ab, H_a)
    assert np.max(np.abs(z)) < 5.0 and np.mean(z * z) < 1.6
    # more detections per history: the band holds sin(psi_max) of the sphere
    assert len(rf) / (16 * N) > 5 * len(ra) / H_a
