"""Pins for the oracle's ordered-subset, dual-matrix and additive-term EM
(paper Sec. 5.3-5.4) and for the primary-only tally.

One subset with the same matrix and no additive term is ML-EM; a
consistent system with an additive term has the true image as a fixed
point; OSEM converges on a consistent invertible system; the primary-only
matrix is the unscattered part of the full one (entry-wise below it, equal
when nothing scatters)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2105_13324_gb300 import phantoms as P


def test_subset_rows_partition_all_rows():
    n_rows, rpv = 12 * 7, 7
    for n_sub in (1, 2, 5, 12):
        rows = np.concatenate([oracle.subset_rows(n_rows, rpv, n_sub, s) for s in range(n_sub)])
        np.testing.assert_array_equal(np.sort(rows), np.arange(n_rows))
        views = oracle.subset_rows(n_rows, rpv, n_sub, 1 % n_sub) // rpv
        assert np.all(views % n_sub == 1 % n_sub)


def _system(seed, m=60, n=20):
    rng = np.random.default_rng(seed)
    a = sp.random(m, n, density=0.3, random_state=rng, format="csr") + sp.csr_matrix(
        (np.full(m, 0.1), (np.arange(m), np.arange(m) % n)), shape=(m, n))
    return sp.csr_matrix(a), rng


def test_one_subset_is_mlem():
    a, rng = _system(1)
    y = rng.poisson(a @ rng.uniform(0, 2, a.shape[1])).astype(float)
    x0 = oracle.mlem_init(a, y)
    want = oracle.mlem(a, y, x0, 7)
    got = oracle.osem(a, a, [np.arange(a.shape[0])], y, x0, 7)
    np.testing.assert_allclose(got, want, rtol=1e-14)
    got0 = oracle.osem(a, a, [np.arange(a.shape[0])], y, x0, 7, add=np.zeros(a.shape[0]))
    np.testing.assert_allclose(got0, want, rtol=1e-14)


def test_additive_term_fixed_point_and_subset_convergence():
    rng = np.random.default_rng(2)
    n, views, rpv = 8, 6, 8
    a = sp.csr_matrix(np.vstack([np.eye(n) * 2.0 + rng.uniform(0.0, 0.2, (n, n)) for _ in range(views)]))
    x_true = rng.uniform(0.5, 2.0, n)
    add = rng.uniform(0.1, 0.5, a.shape[0])
    y = a @ x_true + add
    subsets = [oracle.subset_rows(a.shape[0], rpv, 3, s) for s in range(3)]
    np.testing.assert_allclose(oracle.osem(a, a, subsets, y, x_true, 1, add=add), x_true, rtol=1e-12)
    x = oracle.osem(a, a, subsets, y, np.ones(n), 400, add=add)
    np.testing.assert_allclose(x, x_true, rtol=1e-8)


def test_dual_matrix_with_equal_matrices_is_osem():
    a, rng = _system(3, m=8 * 6, n=12)
    y = rng.poisson(a @ rng.uniform(0, 2, 12)).astype(float)
    subsets = [oracle.subset_rows(a.shape[0], 8, 2, s) for s in range(2)]
    x0 = np.ones(12)
    b = a.copy()
    np.testing.assert_allclose(oracle.osem(a, b, subsets, y, x0, 5), oracle.osem(a, a, subsets, y, x0, 5), rtol=1e-15)


def test_primary_only_matrix_is_the_unscattered_part():
    w = P.workload("water32")
    H = 2_000_000
    full = oracle.build_system(oracle.Problem(w.phantom, w.geometry), w.seed, H)[1]
    prim = oracle.build_system(oracle.Problem(w.phantom, w.geometry, primary_only=True), w.seed, H)[1]
    assert prim.sum() < full.sum() and prim.sum() > 0.5 * full.sum()
    d = (full - prim)
    assert d.min() >= 0
    # nothing scatters in vacuum: both tallies agree
    ph = P.vacuum_phantom(4, 1.0)
    g = P.Geometry(n_views=8, arc_deg=360.0, n_bins_u=32, n_bins_v=32, bin_mm=4.0,
                   radius_mm=P.front_face_radius(4, 1.0), hole_len_mm=5.0, hole_diam_mm=1.5)
    f0 = oracle.build_system(oracle.Problem(ph, g), 3, 300_000)[1]
    p0 = oracle.build_system(oracle.Problem(ph, g, primary_only=True), 3, 300_000)[1]
    assert (f0 != p0).nnz == 0 and f0.nnz > 0


def test_voxels_outside_a_subset_keep_their_value():
    # voxel 2 is seen only by rows of subset 0: subset 1 must not change it
    a = sp.csr_matrix(np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 0.0], [1.0, 1.0, 0.0], [0.0, 2.0, 0.0]]))
    y = np.array([2.0, 1.0, 3.0, 2.0])
    x0 = np.array([1.0, 1.0, 5.0])
    sub1 = np.array([2, 3])            # rows that do not see voxel 2
    x = oracle.osem(a, a, [sub1], y, x0, 1)
    assert x[2] == 5.0
