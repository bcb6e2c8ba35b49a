"""Partitioned ML-EM algebra: the multi-GPU split of Eq. (MLEM), run
sequentially over the parts on the CPU.

A reconstruction too large for one device splits one ML-EM iteration in one
of two ways; either must give the image of the whole iteration:
- rows by views: each part projects x through its own rows, forms its
  ratios y_j / q_j and back-projects them into a partial image; the partial
  images summed (one all-reduce of N values per iteration) give A^T r, and
  the multiplicative update is replicated;
- voxels: each part projects its own voxels; the partial projections summed
  (one all-reduce of M values) give q, and each part updates its own voxels
  with its own columns of A^T.
The sensitivity s_v = sum_j A_jv splits the same way.  The library itself
runs independent acquisitions per rank (no collective); this pins the
algebra of the split a single large reconstruction would use.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2105_13324_gb300 import phantoms as P


@pytest.fixture(scope="module")
def problem():
    w = P.workload("torso64")
    pr = oracle.Problem(w.phantom, w.geometry)
    a, c, nv, fates = oracle.build_system(pr, w.seed, 3_000_000)
    x_true = np.asarray(w.phantom.activity, np.float64).ravel()
    q = a @ x_true
    rng = np.random.Generator(np.random.Philox(11))
    y = rng.poisson(q * (2e5 / max(q.sum(), 1e-30))).astype(np.float64)
    rows_per_view = w.geometry.n_bins_u * w.geometry.n_bins_v
    return sp.csr_matrix(a), y, rows_per_view, w.geometry.n_views


def _ratio(y, q):
    r = np.zeros_like(q)
    np.divide(y, q, out=r, where=q > 0)
    return r


def _step_by_views(a, y, x, view_parts, rows_per_view):
    b = np.zeros_like(x)
    s = np.zeros_like(x)
    for views in view_parts:
        rows = (np.asarray(views)[:, None] * rows_per_view + np.arange(rows_per_view)[None, :]).ravel()
        ap = a[rows]
        b += ap.T @ _ratio(y[rows], ap @ x)   # partial back-projection, summed across parts
        s += np.asarray(ap.sum(axis=0)).ravel()
    out = np.zeros_like(x)
    np.divide(x * b, s, out=out, where=s > 0)
    return out


def _step_by_voxels(a, y, x, col_parts):
    ac = sp.csc_matrix(a)
    q = np.zeros(a.shape[0])
    for cols in col_parts:
        q += ac[:, cols] @ x[cols]            # partial projection, summed across parts
    r = _ratio(y, q)
    out = np.zeros_like(x)
    for cols in col_parts:
        ag = ac[:, cols]
        s = np.asarray(ag.sum(axis=0)).ravel()
        upd = np.zeros(len(cols))
        np.divide(x[cols] * (ag.T @ r), s, out=upd, where=s > 0)
        out[cols] = upd
    return out


@pytest.mark.parametrize("n_parts,interleaved", [(2, False), (3, True), (7, False), (60, False)])
def test_view_partitioned_iterations_equal_the_whole(problem, n_parts, interleaved):
    a, y, rpv, n_views = problem
    views = np.arange(n_views)
    parts = [views[p::n_parts] for p in range(n_parts)] if interleaved else np.array_split(views, n_parts)
    x = oracle.mlem_init(a, y)
    x_part = x.copy()
    x_whole = oracle.mlem(a, y, x, 5)
    for _ in range(5):
        x_part = _step_by_views(a, y, x_part, parts, rpv)
    np.testing.assert_allclose(x_part, x_whole, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("n_parts", [2, 5, 16])
def test_voxel_partitioned_iterations_equal_the_whole(problem, n_parts):
    a, y, rpv, n_views = problem
    n = a.shape[1]
    rng = np.random.default_rng(n_parts)
    cols = rng.permutation(n)                  # any split of the voxels
    parts = [np.sort(c) for c in np.array_split(cols, n_parts)]
    x = oracle.mlem_init(a, y)
    x_part = x.copy()
    x_whole = oracle.mlem(a, y, x, 5)
    for _ in range(5):
        x_part = _step_by_voxels(a, y, x_part, parts)
    np.testing.assert_allclose(x_part, x_whole, rtol=1e-12, atol=1e-300)


def test_a_lost_partial_changes_the_image(problem):
    # the check has teeth: dropping one part's back-projection partial
    a, y, rpv, n_views = problem
    views = np.arange(n_views)
    parts = np.array_split(views, 4)
    x = oracle.mlem_init(a, y)
    good = _step_by_views(a, y, x, parts, rpv)
    bad = _step_by_views(a, y, x, parts[:3], rpv)
    assert not np.allclose(good, bad, rtol=1e-6)
