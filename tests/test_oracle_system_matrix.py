"""Pins for the oracle's system matrix and ML-EM start image.

Eq. (IMC) of Sec. 5.1 defines T_ij as the probability that a photon emitted
in voxel i is detected in bin j; the Monte Carlo estimate divides each
voxel's detections by the histories started there, A = C diag(1/n_v).  The
pins below fix that normalisation from outside the oracle's code: by hand
on a small count matrix, and statistically against the collimator's exact
acceptance integral in vacuum with only two or three histories per voxel,
where a normalisation off by one history (1/(n_v + 1)) shifts the estimate
by a third or more.

The start image of ML-EM (Eq. (MLEM) is silent on it) is read as the uniform
image on the voxels with positive sensitivity whose projection carries the
measured total count; it is fixed by hand on a three-voxel system and by that
property on a random one.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy import integrate

import oracle
from paper_2105_13324_gb300 import phantoms as P


def test_system_matrix_by_hand():
    # columns: n_v = 1, 2, 3, 0 (a voxel without histories has no counts)
    c = sp.csc_matrix(np.array([[1, 0, 2, 0],
                                [0, 1, 1, 0],
                                [1, 2, 0, 0]], dtype=np.int64))
    n_v = np.array([1, 2, 3, 0])
    want = np.array([[1.0, 0.0, 2.0 / 3.0, 0.0],
                     [0.0, 0.5, 1.0 / 3.0, 0.0],
                     [1.0, 1.0, 0.0, 0.0]])
    a = oracle.system_matrix(c, n_v)
    assert a.shape == (3, 4)
    np.testing.assert_array_equal(a.toarray(), want)
    # CSR with sorted column indices, as the oracle's ML-EM expects
    assert sp.isspmatrix_csr(a) and a.has_sorted_indices


def test_system_matrix_of_an_empty_tally():
    a = oracle.system_matrix(sp.csc_matrix((5, 3), dtype=np.int64), np.array([0, 4, 1]))
    assert a.shape == (5, 3) and a.nnz == 0


def _acceptance_per_view(L, d):
    """Per-view detection probability of an unattenuated isotropic emitter
    behind an ideal parallel-hole collimator (hole length L, diameter d):
    1/2 int_0^1 f(x) t / (1 + t^2)^(3/2) dt/dx dx, t = x d / L, with
    f(x) = (2/pi)(acos x - x sqrt(1 - x^2)) the overlap of the hole's ends."""
    def integrand(x):
        t = x * d / L
        f = (2 / math.pi) * (math.acos(x) - x * math.sqrt(1 - x * x))
        return 0.5 * f * t / (1 + t * t) ** 1.5 * (d / L)

    return integrate.quad(integrand, 0, 1, epsabs=0, epsrel=1e-12)[0]


def test_column_sums_estimate_the_detection_probability_with_few_histories_per_voxel():
    # 24^3 vacuum grid (1 mm voxels), 32 views, a detector far wider than the
    # grid's projection plus the collimator's spread: every voxel's
    # detection probability is 32 p_view, whatever its position.
    n, h, V, B, bin_mm, L, d = 24, 1.0, 32, 48, 4.0, 5.0, 1.5
    ph = P.vacuum_phantom(n, h)
    g = P.Geometry(n_views=V, arc_deg=360.0, n_bins_u=B, n_bins_v=B, bin_mm=bin_mm,
                   radius_mm=P.front_face_radius(n, h), hole_len_mm=L, hole_diam_mm=d, fwhm_mm=0.5)
    pr = oracle.Problem(ph, g)
    N = n ** 3
    p_hist = V * _acceptance_per_view(L, d)
    H = 2 * N + N // 2                      # n_v = 3 for the first half of the voxels, 2 for the rest
    a, c, n_v, fates = oracle.build_system(pr, 11, H, threads=4)
    assert fates[oracle.FATE_ESCAPE] == H
    assert set(np.unique(n_v)) == {2, 3}
    s = oracle.sensitivity(a)
    for k in (2, 3):
        sel = n_v == k
        events = int(c[:, np.flatnonzero(sel)].sum())
        # mean column sum over these voxels estimates p_hist; its standard
        # error follows from the (Poisson) event count
        est = float(s[sel].mean())
        err = p_hist * math.sqrt(1.0 / max(events, 1))
        assert events > 1500
        assert abs(est - p_hist) < 4.0 * err, (k, est, p_hist, err)


def test_mlem_start_image_by_hand():
    # s = (2, 0, 1): voxel 1 is outside the support
    a = sp.csr_matrix(np.array([[1.0, 0.0, 0.5],
                                [1.0, 0.0, 0.5]]))
    y = np.array([4.0, 5.0])
    x0 = oracle.mlem_init(a, y)
    np.testing.assert_array_equal(x0, np.array([3.0, 0.0, 3.0]))   # 9 / 3 on the support


def test_mlem_start_image_projects_to_the_measured_total():
    rng = np.random.default_rng(4)
    a = sp.random(60, 30, density=0.1, random_state=rng, format="csr")
    a = sp.csr_matrix(a.toarray() * (np.arange(30) % 5 != 0))    # every fifth voxel unseen
    y = rng.poisson(5.0, 60).astype(np.float64)
    x0 = oracle.mlem_init(a, y)
    s = np.asarray(a.sum(axis=0)).ravel()
    assert np.all(x0[s == 0] == 0.0)
    sup = x0[s > 0]
    assert np.all(sup == sup[0]) and sup[0] > 0           # uniform on the support
    assert float((a @ x0).sum()) == pytest.approx(float(y.sum()), rel=1e-13)


def test_mlem_start_image_without_sensitivity_is_zero():
    a = sp.csr_matrix((4, 3))
    np.testing.assert_array_equal(oracle.mlem_init(a, np.ones(4)), np.zeros(3))
