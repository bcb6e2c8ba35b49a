"""Forced detection on the GPU against the FP64 oracle (through the C ABI).

- weighted assembly: the oracle's forced-detection events assembled by the
  library equal the oracle's weight sums exactly (integer fixed point);
- FP64 transport + forced copies: the same matrix as the oracle's, entry by
  entry, on a small problem and on the full 128^3 x 120-view geometry (a
  short history range), for all photons and for the unscattered part;
- FP32: the same events up to rounding (totals, views, entries), on the
  small problem and on the full geometry, where the float traversal crosses
  whole cubes of one material per step;
- the matrix drives ML-EM like any other system, and builds are
  reproducible bit for bit (integer weight sums do not depend on the order
  in which events arrive).
"""
import numpy as np
import pytest

import oracle
from paper_2105_13324_gb300 import phantoms as P

from tests.distance_map_ref import distance_map_by_definition

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    return mcspect


def _small():
    ph = P.water_cylinder_phantom(16, 4.0, radius=24.0, shell_outer=(14.0, 12.0, 12.0), wall=5.0)
    c = P.voxel_centres(16, 4.0)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    ph.material = ph.material.copy()
    ph.material[:, (xx - 6.0) ** 2 + yy ** 2 <= 10.0 ** 2] = 2
    ph.rho, ph.z_over_a, ph.z_eff = (np.append(ph.rho, 1.85), np.append(ph.z_over_a, 0.5148),
                                     np.append(ph.z_eff, 13.0))
    g = P.spect_geometry(8, 360.0, 16, 4.0, 16, 4.0, hole_len_mm=20.0, hole_diam_mm=2.0, fwhm_mm=4.0,
                         window_frac=0.5)
    return ph, g


def _csc(mc_sys):
    cp, ri, cnt, nv = mc_sys.export_csc()
    vals, _ = mc_sys.export_values()
    cols = np.repeat(np.arange(len(cp) - 1), np.diff(cp))
    return cols.astype(np.int64) * mc_sys.shape[0] + ri, vals, cnt, nv


def _oracle_fd(ph, g, seed, first, count, primary=False):
    pr = oracle.Problem(ph, g, primary_only=primary, forced_detection=True)
    rows, cols, q, fates = oracle.run_fd(pr, seed, first, count)
    key = cols * pr.n_rows + rows
    order = np.argsort(key, kind="stable")
    ks, qs = key[order], q[order]
    heads = np.flatnonzero(np.r_[True, ks[1:] != ks[:-1]]) if len(ks) else np.zeros(0, np.int64)
    return pr, rows, cols, q, ks[heads], np.add.reduceat(qs, heads) if len(ks) else np.zeros(0, np.int64), fates


def test_weighted_assembly_is_exact(mc):
    ph, g = _small()
    pr, rows, cols, q, uk, sums, _ = _oracle_fd(ph, g, 3, 0, 20000)
    s = mc.mc_system_from_weighted_events(pr.n_rows, pr.n_voxels, rows, cols.astype(np.int32), q, 0, 20000)
    key, vals, cnt, nv = _csc(s)
    assert s.info()["weighted"]
    np.testing.assert_array_equal(key, uk)
    np.testing.assert_array_equal(vals, sums.astype(np.float64) / mc.FD_SCALE)   # exact: integer sums
    np.testing.assert_array_equal(nv, oracle.histories_per_voxel(pr.n_voxels, 0, 20000))
    # CSR holds the same entries
    rp, ci, _ = s.export_csr()
    _, vals_csr = s.export_values()
    rows_r = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    key_r = ci.astype(np.int64) * pr.n_rows + rows_r
    o = np.argsort(key_r)
    np.testing.assert_array_equal(key_r[o], uk)
    np.testing.assert_array_equal(vals_csr[o], vals)
    # column sums drive the sensitivity
    import torch
    sens = torch.zeros(pr.n_voxels, dtype=torch.float64, device="cuda")
    mc.mc_sensitivity(s, sens)
    w = oracle.system_weights(rows, cols, q, pr.n_rows, pr.n_voxels)
    a = oracle.system_matrix(w, nv.astype(np.int64))
    np.testing.assert_allclose(sens.cpu().numpy(), oracle.sensitivity(a), rtol=1e-13, atol=0)
    # empty event list
    e = mc.mc_system_from_weighted_events(pr.n_rows, pr.n_voxels, np.zeros(0), np.zeros(0), np.zeros(0), 0, 10)
    assert e.info()["nnz"] == 0 and e.info()["weighted"]
    with pytest.raises(mc.McError):
        mc.mc_system_from_weighted_events(pr.n_rows, pr.n_voxels, [pr.n_rows], [0], [5], 0, 1)


def _compare_fp64(mc, ph, g, seed, first, count, primary):
    pr, rows, cols, q, uk, sums, fates = _oracle_fd(ph, g, seed, first, count, primary)
    s = mc.mc_build_system_range(ph, g, first, count, seed, precision="fp64", primary_only=primary, forced=True)
    inf = s.info()
    assert inf["weighted"] and inf["n_events"] == len(rows)
    assert inf["fates"] == [int(f) for f in fates]
    key, vals, cnt, nv = _csc(s)
    # identical structure; weight sums equal up to last-bit differences of
    # log/exp/acos between CUDA and the host's libm (a unit of 2^-48 in a sum)
    common, ia, ib = np.intersect1d(key, uk, return_indices=True)
    assert len(common) >= 0.9999 * len(uk) and len(key) <= len(uk) + max(2, len(uk) // 10000)
    want = sums[ib].astype(np.float64) / mc.FD_SCALE
    np.testing.assert_allclose(vals[ia], want, rtol=1e-9, atol=4.0 / mc.FD_SCALE)
    return s, pr


@pytest.mark.parametrize("primary", [False, True])
def test_fp64_forced_detection_matches_oracle_small(mc, primary):
    ph, g = _small()
    _compare_fp64(mc, ph, g, 17, 1000, 3 * 16 ** 3 + 77, primary)


def test_fp64_forced_detection_matches_oracle_full_geometry(mc):
    # the benchmark's 128^3 x 2 mm torso and 120 views over 360 degrees, a
    # range of histories spread over the grid
    w = P.workload("torso128")
    _compare_fp64(mc, w.phantom, w.geometry, 5, 123_456, 4000, False)


def test_fp32_forced_detection_matches_oracle(mc):
    ph, g = _small()
    pr, rows, cols, q, uk, sums, fates = _oracle_fd(ph, g, 9, 0, 4 * 16 ** 3)
    s = mc.mc_build_system(ph, g, 4 * 16 ** 3, 9, precision="fp32", forced=True)
    key, vals, cnt, nv = _csc(s)
    want_total = sums.sum() / mc.FD_SCALE
    # float weights carry ~1e-6 relative rounding (fast exp/log/sincos)
    assert vals.sum() == pytest.approx(want_total, rel=3e-5)
    # per view
    M = pr.n_rows
    rows_g = key % M
    view_g = np.bincount(rows_g // 256, weights=vals, minlength=8)
    view_o = np.bincount((uk % M) // 256, weights=sums / mc.FD_SCALE, minlength=8)
    np.testing.assert_allclose(view_g, view_o, rtol=1e-4)
    # entries: the same events up to float rounding (a rare copy may land in
    # the neighbouring bin)
    common, ia, ib = np.intersect1d(key, uk, return_indices=True)
    assert len(common) >= 0.999 * len(uk)
    rel = np.abs(vals[ia] - sums[ib] / mc.FD_SCALE) / (sums[ib] / mc.FD_SCALE)
    assert np.mean(rel > 1e-3) < 1e-3


def test_fp32_forced_detection_matches_oracle_full_geometry(mc):
    # large homogeneous regions (body, lungs, air): the float traversal's
    # cube steps must give the same transmissions as the oracle's voxel walk
    w = P.workload("torso128")
    first, count = 777_777, 3000
    pr, rows, cols, q, uk, sums, fates = _oracle_fd(w.phantom, w.geometry, 11, first, count)
    s = mc.mc_build_system_range(w.phantom, w.geometry, first, count, 11, precision="fp32", forced=True)
    key, vals, cnt, nv = _csc(s)
    want = sums / mc.FD_SCALE
    assert vals.sum() == pytest.approx(want.sum(), rel=3e-5)
    M = pr.n_rows
    per_view = M // w.geometry.n_views
    view_g = np.bincount((key % M) // per_view, weights=vals, minlength=w.geometry.n_views)
    view_o = np.bincount((uk % M) // per_view, weights=want, minlength=w.geometry.n_views)
    np.testing.assert_allclose(view_g, view_o, rtol=2e-4)
    common, ia, ib = np.intersect1d(key, uk, return_indices=True)
    assert len(common) >= 0.999 * len(uk)
    rel = np.abs(vals[ia] - want[ib]) / want[ib]
    assert np.mean(rel > 1e-3) < 1e-3
    assert np.median(rel) < 5e-5


def test_forced_build_over_several_launches_equals_its_ranges(mc):
    # more histories than one forced-detection launch takes (2^21): the
    # integer weight sums of the launches add up exactly to those of two
    # separate builds of the range's halves
    import scipy.sparse as sp
    ph, g = _small()
    H, m = (1 << 21) + 3_333, 1_234_567

    def mat(s):
        cp, ri, cnt, nv = s.export_csc()
        vals, _ = s.export_values()
        M, N = s.shape
        return (sp.csc_matrix((vals, ri, cp), shape=(M, N)), sp.csc_matrix((cnt.astype(np.int64), ri, cp), shape=(M, N)))

    full = mc.mc_build_system(ph, g, H, 21, precision="fp32", forced=True)
    a = mc.mc_build_system_range(ph, g, 0, m, 21, precision="fp32", forced=True)
    b = mc.mc_build_system_range(ph, g, m, H - m, 21, precision="fp32", forced=True)
    (wf, cf), (wa, ca), (wb, cb) = mat(full), mat(a), mat(b)
    assert (cf != ca + cb).nnz == 0
    assert (wf != wa + wb).nnz == 0
    assert full.info()["fates"] == [x + y for x, y in zip(a.info()["fates"], b.info()["fates"])]


def test_distance_map_matches_its_definition(mc):
    rng = np.random.default_rng(4)
    ph, _ = _small()
    cases = [ph.material]
    # blobs of 3 materials on an odd-shaped grid, a one-material grid (the
    # cap), a single voxel and a one-voxel-thick slab
    z, y, x = np.meshgrid(np.arange(7), np.arange(9), np.arange(23), indexing="ij")
    blob = ((x - 6) ** 2 + (y - 4) ** 2 + (z - 3) ** 2 < 10).astype(np.uint8)
    blob[(x - 17) ** 2 + (y - 2) ** 2 < 5] = 2
    cases += [blob, np.zeros((5, 6, 40), np.uint8), np.zeros((1, 1, 1), np.uint8),
              (x[:3] == 11).astype(np.uint8)[:, :, :]]
    cases.append(rng.integers(0, 2, (6, 5, 4)).astype(np.uint8))
    for mat in cases:
        q = P.Phantom(np.ascontiguousarray(mat), np.array([0.001, 1.0, 1.9]), np.array([0.5, 0.55, 0.52]),
                      np.array([7.6, 7.4, 13.0]), 2.0)
        got = mc.mc_debug_distance_map(q)
        np.testing.assert_array_equal(got, distance_map_by_definition(mat))


def test_forced_system_drives_mlem_and_is_reproducible(mc):
    import torch
    ph, g = _small()
    H = 8 * 16 ** 3
    s1 = mc.mc_build_system(ph, g, H, 4, precision="fp32", forced=True)
    s2 = mc.mc_build_system(ph, g, H, 4, precision="fp32", forced=True)
    k1, v1, _, _ = _csc(s1)
    k2, v2, _, _ = _csc(s2)
    np.testing.assert_array_equal(k1, k2)
    np.testing.assert_array_equal(v1, v2)
    cp, ri, _, nv = s1.export_csc()
    w = __import__("scipy.sparse", fromlist=["csc_matrix"]).csc_matrix((v1, ri, cp), shape=s1.shape)
    a = oracle.system_matrix(w, nv.astype(np.int64))
    y = P.poisson_counts(a @ ph.activity.ravel().astype(np.float64), 2e5, 3)
    yd = torch.as_tensor(y).cuda()
    x = torch.zeros(s1.shape[1], dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(s1, yd, x)
    mc.mlem_iterate(s1, yd, x, 20)
    want = oracle.mlem(a, y, oracle.mlem_init(a, y), 20)
    got = x.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5
    # weighted systems keep float values and have no ordered subsets
    with pytest.raises(mc.McError):
        s1.set_value_type("f16", allow_rounding=True)
    with pytest.raises(mc.McError):
        mc.mc_system_subset(s1, 256, 2, 0)


def test_forced_direction_primary_matches_oracle(mc):
    # FP64: the same histories and draws as the oracle, so the same
    # detections; every event weighs rint(sin(psi) 2^48): exact sums
    ph, g = _small()
    first, count = 500, 40 * 16 ** 3
    pr = oracle.Problem(ph, g, primary_only=True, forced_direction=True)
    rows, cols, q, fates = oracle.run_fd(pr, 13, first, count)
    want = oracle.system_weights(rows, cols, q, pr.n_rows, pr.n_voxels)
    s = mc.mc_build_system_range(ph, g, first, count, 13, precision="fp64", primary_only=True, forced_direction=True)
    inf = s.info()
    assert inf["weighted"] and inf["fates"] == [int(f) for f in fates]
    cp, ri, cnt, nv = s.export_csc()
    vals, _ = s.export_values()
    np.testing.assert_array_equal(cp, want.indptr)
    np.testing.assert_array_equal(ri, want.indices)
    np.testing.assert_array_equal(vals, want.data)
    band = oracle.direction_band(pr)
    np.testing.assert_array_equal(vals, cnt * (round(band * mc.FD_SCALE) / mc.FD_SCALE))
    # per-history traces agree too (same draws, same fates)
    rec_g = mc.mc_trace_histories(ph, g, 13, first, 4000, primary_only=True, forced_direction=True)
    rec_o = oracle.trace(pr, 13, first, 4000)
    for f in ("fate", "n_events", "n_virtual", "n_real", "n_compton", "n_draws"):
        np.testing.assert_array_equal(rec_g[f], rec_o[f])
    # FP32: the same detections up to rounding
    s32 = mc.mc_build_system_range(ph, g, first, count, 13, precision="fp32", primary_only=True,
                                   forced_direction=True)
    rp, _, c32 = s32.export_csr()
    rows_g = np.bincount(np.repeat(np.arange(pr.n_rows), np.diff(rp)), weights=c32.astype(np.float64),
                         minlength=pr.n_rows)
    rows_o = np.bincount(rows, minlength=pr.n_rows).astype(np.float64)
    assert np.all(np.abs(rows_g - rows_o) <= 3 * np.sqrt(rows_g + rows_o) + 1e-9)
    assert abs(rows_g.sum() - rows_o.sum()) <= 0.01 * rows_o.sum()
    # forced direction goes with the primary tally only
    with pytest.raises(mc.McError):
        mc.mc_build_system(ph, g, 100, 1, forced_direction=True)


def test_forced_detection_in_vacuum_and_empty_cases(mc):
    # vacuum: every copy crosses the grid unattenuated; the FP64 build equals
    # the oracle's (no collisions: emission copies only)
    ph = P.vacuum_phantom(8, 4.0)
    g = P.spect_geometry(6, 360.0, 16, 4.0, 8, 4.0, hole_len_mm=20.0, hole_diam_mm=2.0, fwhm_mm=2.0)
    pr = oracle.Problem(ph, g, forced_detection=True)
    rows, cols, q, fates = oracle.run_fd(pr, 2, 0, 3000)
    want = oracle.system_weights(rows, cols, q, pr.n_rows, pr.n_voxels)
    s = mc.mc_build_system(ph, g, 3000, 2, precision="fp64", forced=True)
    assert s.info()["fates"] == [0, 0, 3000, 0]
    cp, ri, _, _ = s.export_csc()
    vals, _ = s.export_values()
    np.testing.assert_array_equal(cp, want.indptr)
    np.testing.assert_array_equal(ri, want.indices)
    np.testing.assert_allclose(vals, want.data, rtol=1e-12, atol=2.0 / mc.FD_SCALE)
    # one history; a history range starting anywhere
    s1 = mc.mc_build_system_range(ph, g, 123_456_789, 1, 2, precision="fp64", forced=True)
    r1, c1, q1, _ = oracle.run_fd(pr, 2, 123_456_789, 1)
    assert s1.info()["n_events"] == len(r1) == len(np.unique(r1))
    with pytest.raises(mc.McError):
        mc.mc_build_system(ph, g, 0, 2, forced=True)
