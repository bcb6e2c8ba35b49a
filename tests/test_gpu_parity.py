"""GPU path vs the CPU oracle, element by element, through the C ABI.

Transport: per-history traces in FP64 verification mode (>= 99.99 % of
histories identical), bit-exact count matrices from the same histories,
FP32 tallies within 3 sigma of the FP64 oracle on the same streams.
Assembly: bit-exact CSC/CSR from an oracle event list.  Reconstruction:
projectors and ML-EM in FP32 against the FP64 oracle on the same matrix
(relative L2 <= 1e-5).  Edge cases: empty and single-event matrices,
ragged sizes, a vacuum phantom.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

MLEM_TOL = 1e-5   # relative L2, FP32 GPU vs FP64 oracle on the same matrix


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    return mcspect


def _dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _compare_traces(g, o):
    same = ((g["fate"] == o["fate"]) & (g["n_virtual"] == o["n_virtual"]) & (g["n_real"] == o["n_real"])
            & (g["n_compton"] == o["n_compton"]) & (g["n_draws"] == o["n_draws"])
            & (g["n_events"] == o["n_events"]) & np.all(g["event_row"] == o["event_row"], axis=1)
            & (np.abs(g["e_final_kev"] - o["e_final_kev"]) <= 1e-12 * o["e_final_kev"]))
    return same


# ---------------------------------------------------------------------------
# transport
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,first,count", [("water32", 0, 2_000_000), ("torso64", 7_777_777, 300_000),
                                              ("torso128", 987_654_321, 200_000)])
def test_fp64_trace_matches_oracle(mc, name, first, count):
    w = P.workload(name)
    g = mc.mc_trace_histories(w.phantom, w.geometry, w.seed, first, count, precision="fp64")
    o = oracle.trace(oracle.Problem(w.phantom, w.geometry), w.seed, first, count)
    same = _compare_traces(g, o)
    frac = same.mean()
    bad = np.nonzero(~same)[0][:10]
    assert frac >= 0.9999, (frac, [(int(first + i), g[i], o[i]) for i in bad])
    assert g["n_events"].sum() > 0


def test_fp64_matrix_is_bit_exact(mc):
    w = P.workload("water32")
    pr = oracle.Problem(w.phantom, w.geometry)
    H = w.n_histories
    sysm = mc.mc_build_system(w.phantom, w.geometry, H, w.seed, precision="fp64")
    info = sysm.info()
    a_orc, c_orc, nv_orc, fates = oracle.build_system(pr, w.seed, H)
    assert info["fates"] == [int(f) for f in fates]
    cp, ri, cnt, nv = sysm.export_csc()
    np.testing.assert_array_equal(nv, nv_orc)
    np.testing.assert_array_equal(cp, c_orc.indptr)
    np.testing.assert_array_equal(ri, c_orc.indices)
    np.testing.assert_array_equal(cnt, c_orc.data)
    rp, ci, cnt_r = sysm.export_csr()
    c_csr = sp.csr_matrix(c_orc)
    c_csr.sort_indices()
    np.testing.assert_array_equal(rp, c_csr.indptr)
    np.testing.assert_array_equal(ci, c_csr.indices)
    np.testing.assert_array_equal(cnt_r, c_csr.data)
    assert info["n_events"] == int(c_orc.sum())


def _tally_close(c_gpu, c_orc):
    d = np.abs(c_gpu - c_orc)
    lim = 3.0 * np.sqrt(c_gpu + c_orc) + 1e-12
    return np.all((d <= lim) | (d == 0))


@pytest.mark.parametrize("name,H", [("water32", 2_000_000), ("torso64", 3_000_000)])
def test_fp32_tallies_within_3_sigma_of_oracle(mc, name, H):
    w = P.workload(name)
    pr = oracle.Problem(w.phantom, w.geometry)
    sysm = mc.mc_build_system(w.phantom, w.geometry, H, w.seed, precision="fp32")
    cp, ri, cnt, nv = sysm.export_csc()
    c_gpu = sp.csc_matrix((cnt.astype(np.float64), ri, cp), shape=(pr.n_rows, pr.n_voxels))
    _, c_orc, nv_orc, fates = oracle.build_system(pr, w.seed, H)
    c_orc = c_orc.astype(np.float64)
    np.testing.assert_array_equal(nv, nv_orc)
    info = sysm.info()
    assert sum(info["fates"]) == H and info["fates"][3] == 0
    for f in range(3):   # fates: same streams, so nearly identical
        assert abs(info["fates"][f] - int(fates[f])) <= 3 * np.sqrt(info["fates"][f] + int(fates[f])) + 1
    assert _tally_close(np.asarray(c_gpu.sum(axis=0)).ravel(), np.asarray(c_orc.sum(axis=0)).ravel())
    assert _tally_close(np.asarray(c_gpu.sum(axis=1)).ravel(), np.asarray(c_orc.sum(axis=1)).ravel())
    _entries_within_3_sigma(c_gpu, c_orc)
    # shared streams: the vast majority of entries agree exactly
    assert abs(c_gpu - c_orc).sum() <= 0.01 * c_orc.sum() + 5


def _entries_within_3_sigma(c_gpu, c_orc):
    """Every non-zero of either matrix: |C_gpu - C_orc| <= 3 sqrt(C_gpu + C_orc)."""
    diff = (c_gpu - c_orc).tocoo()
    both = (c_gpu + c_orc).tocsr()
    lim = 3.0 * np.sqrt(np.asarray(both[diff.row, diff.col]).ravel())
    assert np.all(np.abs(diff.data) <= lim + 1e-12)


def test_fp32_bench_workload_sample_within_3_sigma(mc):
    # the benchmark's 128^3 torso, 120 views: a range of 4e6 histories from
    # the middle of the benchmark's 1e9, through the same plan-build path
    # and launch configuration, against the oracle on the same range
    w = P.workload("torso128")
    pr = oracle.Problem(w.phantom, w.geometry)
    first, count = 500_000_000, 4_000_000
    plan = mc.Plan(w.phantom, w.geometry, "fp32")
    sysm = plan.build(first, count, w.seed)
    cp, ri, cnt, nv = sysm.export_csc()
    c_gpu = sp.csc_matrix((cnt.astype(np.float64), ri, cp), shape=(pr.n_rows, pr.n_voxels))
    rows, cols, fates = oracle.run(pr, w.seed, first, count)
    c_orc = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels).astype(np.float64)
    np.testing.assert_array_equal(nv, oracle.histories_per_voxel(pr.n_voxels, first, count))
    info = sysm.info()
    for f in range(3):
        assert abs(info["fates"][f] - int(fates[f])) <= 3 * np.sqrt(info["fates"][f] + int(fates[f])) + 1
    assert _tally_close(np.asarray(c_gpu.sum(axis=1)).ravel(), np.asarray(c_orc.sum(axis=1)).ravel())
    assert _tally_close(np.asarray(c_gpu.sum(axis=0)).ravel(), np.asarray(c_orc.sum(axis=0)).ravel())
    _entries_within_3_sigma(c_gpu, c_orc)
    assert abs(c_gpu - c_orc).sum() <= 0.01 * c_orc.sum() + 5
    plan.free()


def test_fp64_compton_sampler_matches_oracle(mc):
    c_g, e_g = mc.mc_debug_kn(140.5, 21, 200_000, precision="fp64")
    c_o, e_o, _ = oracle.kn_sample(140.5, 21, 200_000)
    np.testing.assert_array_equal(c_g, c_o)
    np.testing.assert_allclose(e_g, e_o, rtol=1e-15)


def test_fp32_compton_sampler_follows_klein_nishina(mc):
    from scipy import stats
    c_g, e_g = mc.mc_debug_kn(140.5, 22, 400_000, precision="fp32")
    c_o, e_o, _ = oracle.kn_sample(140.5, 22, 400_000)
    # same streams: the 23-bit uniforms round differently only near rejection edges
    assert np.mean(np.abs(c_g - c_o) < 1e-6) > 0.999
    assert stats.ks_2samp(c_g, c_o).pvalue > 1e-3


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_beam_transmission_matches_oracle(mc, precision):
    ph = P.slab_phantom(40, 4.0, P.WATER, 96.0, (P.BONE,))
    g = P.spect_geometry(1, 180.0, 8, 4.0, 40, 4.0)
    pr = oracle.Problem(ph, g)
    p0, d = (-80.0 + 1e-9, 0.5, 0.5), (1.0, 0.0, 0.0)
    n = 400_000
    got = mc.mc_debug_beam(ph, g, 5, n, p0, d, 140.5, precision=precision)
    want = oracle.beam(pr, 5, n, p0, d, 140.5)
    if precision == "fp64":
        assert got == want
    else:
        assert abs(got - want) <= 3 * np.sqrt(want) + 1


def test_vacuum_phantom_only_collimator_acceptance(mc):
    ph = P.vacuum_phantom(4, 1.0)
    g = P.Geometry(n_views=8, arc_deg=360.0, n_bins_u=64, n_bins_v=64, bin_mm=4.0,
                   radius_mm=P.front_face_radius(4, 1.0), hole_len_mm=5.0, hole_diam_mm=1.5, fwhm_mm=0.5)
    pr = oracle.Problem(ph, g)
    H = 500_000
    sysm = mc.mc_build_system(ph, g, H, 9, precision="fp64")
    _, c_orc, _, fates = oracle.build_system(pr, 9, H)
    cp, ri, cnt, _ = sysm.export_csc()
    np.testing.assert_array_equal(cnt, c_orc.data)
    np.testing.assert_array_equal(ri, c_orc.indices)
    assert sysm.info()["fates"][2] == H


def test_history_ranges_add_up(mc):
    w = P.workload("torso64")
    H, m = 1_000_000, 377_777
    full = mc.mc_build_system(w.phantom, w.geometry, H, w.seed, precision="fp32")
    a = mc.mc_build_system_range(w.phantom, w.geometry, 0, m, w.seed, precision="fp32")
    b = mc.mc_build_system_range(w.phantom, w.geometry, m, H - m, w.seed, precision="fp32")
    M, N = full.shape

    def mat(s):
        cp, ri, cnt, nv = s.export_csc()
        return sp.csc_matrix((cnt.astype(np.int64), ri, cp), shape=(M, N)), nv.astype(np.int64)

    cf, nf = mat(full)
    ca, na = mat(a)
    cb, nb = mat(b)
    assert (cf != ca + cb).nnz == 0
    np.testing.assert_array_equal(nf, na + nb)


def test_build_over_several_launches_equals_its_ranges(mc):
    # more histories than one transport launch takes (2^30 for this
    # collimator): the launches' histories, escape queues and events must
    # add up to the same matrix as two separate builds of the range's halves
    w = P.workload("torso64")
    H, m = (1 << 30) + 54_321, 600_000_001
    full = mc.mc_build_system(w.phantom, w.geometry, H, 3, precision="fp32")
    a = mc.mc_build_system_range(w.phantom, w.geometry, 0, m, 3, precision="fp32")
    b = mc.mc_build_system_range(w.phantom, w.geometry, m, H - m, 3, precision="fp32")
    M, N = full.shape

    def mat(s):
        cp, ri, cnt, nv = s.export_csc()
        return sp.csc_matrix((cnt.astype(np.int64), ri, cp), shape=(M, N)), nv.astype(np.int64)

    cf, nf = mat(full)
    ca, na = mat(a)
    cb, nb = mat(b)
    assert (cf != ca + cb).nnz == 0
    np.testing.assert_array_equal(nf, na + nb)
    assert full.info()["fates"] == [x + y for x, y in zip(a.info()["fates"], b.info()["fates"])]


# ---------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_rows,n_cols,n_events,seed", [
    (37, 23, 0, 1), (37, 23, 1, 2), (1, 1, 1000, 3), (5000, 3001, 123_457, 4), (65537, 40000, 2_000_003, 5)])
def test_assembly_from_events_is_bit_exact(mc, n_rows, n_cols, n_events, seed):
    rng = np.random.default_rng(seed)
    rows = rng.integers(0, n_rows, n_events).astype(np.int32)
    cols = (rng.zipf(1.3, n_events) % n_cols).astype(np.int32)
    sysm = mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, 10 * n_cols + 3)
    want = oracle.system_counts(rows, cols, n_rows, n_cols)
    cp, ri, cnt, nv = sysm.export_csc()
    np.testing.assert_array_equal(cp, want.indptr)
    np.testing.assert_array_equal(ri, want.indices)
    np.testing.assert_array_equal(cnt, want.data)
    np.testing.assert_array_equal(nv, oracle.histories_per_voxel(n_cols, 0, 10 * n_cols + 3))
    rp, ci, cr = sysm.export_csr()
    wr = sp.csr_matrix(want)
    wr.sort_indices()
    np.testing.assert_array_equal(rp, wr.indptr)
    np.testing.assert_array_equal(ci, wr.indices)
    np.testing.assert_array_equal(cr, wr.data)
    info = sysm.info()
    assert info["nnz"] == want.nnz and info["n_events"] == n_events
    assert info["max_count"] == (int(want.data.max()) if want.nnz else 0)


def _bucket_case(kind):
    """Events for the assembly cases below: (n_rows, n_cols, rows, cols)."""
    rng = np.random.Generator(np.random.Philox(100 + len(kind)))
    if kind in ("uniform", "uniform_large"):
        n_rows, n_cols, n = (5003, 3001, 20_011) if kind == "uniform" else (300_007, 200_003, 1_000_003)
        rows = rng.integers(0, n_rows, n)
        cols = rng.integers(0, n_cols, n)
        dup = rng.choice(n, n // 10, replace=False)          # repeated events: counts above 1
        rows, cols = np.concatenate([rows, rows[dup], rows[dup[:n // 50]]]), np.concatenate([cols, cols[dup], cols[dup[:n // 50]]])
    elif kind in ("column_of_64", "column_of_65"):
        n_rows, n_cols = 4001, 2003
        rows = rng.integers(0, n_rows, 8000)
        cols = rng.integers(0, n_cols, 8000)
        cols[cols == 17] = 18
        extra = 64 if kind == "column_of_64" else 65
        rows = np.concatenate([rows, rng.choice(n_rows, extra, replace=False)])
        cols = np.concatenate([cols, np.full(extra, 17)])
    else:  # one long row over short columns
        n_rows, n_cols = 4001, 2003
        rows = np.concatenate([rng.integers(0, n_rows, 8000), np.full(300, 11)])
        cols = np.concatenate([rng.integers(0, n_cols, 8000), rng.choice(n_cols, 300, replace=False)])
    return n_rows, n_cols, rows.astype(np.int32), cols.astype(np.int32)


@pytest.mark.parametrize("kind,buckets", [("uniform", True), ("uniform_large", True), ("column_of_64", True),
                                          ("column_of_65", False), ("long_row", False)])
def test_assembly_by_buckets_and_its_fallbacks_is_bit_exact(mc, kind, buckets):
    # unweighted events whose columns hold at most 64 events and rows at
    # most 64 entries are assembled by column and row buckets; a longer
    # column, or a longer row found after the CSC was made, falls back to the
    # radix sort.  Every case equals the oracle's matrix exactly.
    n_rows, n_cols, rows, cols = _bucket_case(kind)
    want = oracle.system_counts(rows, cols, n_rows, n_cols)
    longest_col = int(np.bincount(cols, minlength=n_cols).max())
    longest_row = int(np.diff(sp.csr_matrix(want).indptr).max())
    assert (longest_col <= 64 and longest_row <= 64) == buckets
    H = 7 * n_cols + 5
    sysm = mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, H)
    cp, ri, cnt, nv = sysm.export_csc()
    np.testing.assert_array_equal(cp, want.indptr)
    np.testing.assert_array_equal(ri, want.indices)
    np.testing.assert_array_equal(cnt, want.data)
    np.testing.assert_array_equal(nv, oracle.histories_per_voxel(n_cols, 0, H))
    rp, ci, cr = sysm.export_csr()
    wr = sp.csr_matrix(want)
    wr.sort_indices()
    np.testing.assert_array_equal(rp, wr.indptr)
    np.testing.assert_array_equal(ci, wr.indices)
    np.testing.assert_array_equal(cr, wr.data)
    info = sysm.info()
    assert info["nnz"] == want.nnz and info["n_events"] == len(rows)
    assert info["max_count"] == int(want.data.max())
    import torch
    s = torch.zeros(n_cols, dtype=torch.float64, device="cuda")
    mc.mc_sensitivity(sysm, s)
    np.testing.assert_allclose(s.cpu().numpy(), oracle.sensitivity(oracle.system_matrix(want, nv)), rtol=1e-13)
    sysm.free()


# ---------------------------------------------------------------------------
# projectors and ML-EM (oracle matrix uploaded as events)
# ---------------------------------------------------------------------------
def _oracle_problem(name, H, seed_shift=0):
    w = P.workload(name)
    pr = oracle.Problem(w.phantom, w.geometry)
    rows, cols, _ = oracle.run(pr, w.seed + seed_shift, 0, H)
    c = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
    nv = oracle.histories_per_voxel(pr.n_voxels, 0, H)
    a = oracle.system_matrix(c, nv)
    return w, pr, rows, cols, a


@pytest.fixture(scope="module")
def torso_small(mc):
    w, pr, rows, cols, a = _oracle_problem("torso64", 20_000_000)
    _, _, _, _, a_truth = _oracle_problem("torso64", 20_000_000, seed_shift=1000)
    ybar = a_truth @ w.phantom.activity.ravel().astype(np.float64)
    y = P.poisson_counts(ybar, w.total_counts, w.noise_seed)
    sysm = mc.mc_system_from_events(pr.n_rows, pr.n_voxels, rows, cols.astype(np.int32), 0, 20_000_000)
    return w, pr, a, y, sysm


def test_projectors_match_oracle(mc, torso_small):
    import torch
    w, pr, a, y, sysm = torso_small
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 2.0, pr.n_voxels).astype(np.float32)
    q = torch.zeros(pr.n_rows, dtype=torch.float32, device="cuda")
    mc.mc_project(sysm, _dev(x), q)
    want_q = a @ x.astype(np.float64)
    assert _rel_l2(q.cpu().numpy(), want_q) < 1e-6
    np.testing.assert_allclose(q.cpu().numpy(), want_q, rtol=1e-5, atol=1e-6 * want_q.max())
    r = rng.uniform(0.0, 2.0, pr.n_rows).astype(np.float32)
    b = torch.zeros(pr.n_voxels, dtype=torch.float32, device="cuda")
    mc.mc_backproject(sysm, _dev(r), b)
    want_b = a.T @ r.astype(np.float64)
    assert _rel_l2(b.cpu().numpy(), want_b) < 1e-6
    s = torch.zeros(pr.n_voxels, dtype=torch.float64, device="cuda")
    mc.mc_sensitivity(sysm, s)
    np.testing.assert_allclose(s.cpu().numpy(), oracle.sensitivity(a), rtol=1e-13)


def test_mlem_matches_oracle(mc, torso_small):
    import torch
    w, pr, a, y, sysm = torso_small
    yd = _dev(y)
    x = torch.zeros(pr.n_voxels, dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(sysm, yd, x)
    x0 = oracle.mlem_init(a, y)
    assert _rel_l2(x.cpu().numpy(), x0) < 1e-7
    ll = mc.mlem_iterate(sysm, yd, x, w.mlem_iters, loglik=True)
    xo, llo = oracle.mlem(a, y, x0, w.mlem_iters, with_loglik=True)
    err = _rel_l2(x.cpu().numpy(), xo)
    assert err <= MLEM_TOL, err
    np.testing.assert_allclose(ll, llo, rtol=1e-6)
    assert np.all(x.cpu().numpy() >= 0)
    # continuing in two calls equals one call of the summed length
    x2 = torch.zeros_like(x)
    mc.mc_mlem_init(sysm, yd, x2)
    mc.mlem_iterate(sysm, yd, x2, 20)
    mc.mlem_iterate(sysm, yd, x2, w.mlem_iters - 20)
    assert torch.equal(x2, x)


def test_mlem_on_degenerate_systems(mc):
    import torch
    # empty matrix: every voxel has zero sensitivity -> zeros, no NaN
    s0 = mc.mc_system_from_events(10, 7, np.zeros(0, np.int32), np.zeros(0, np.int32), 0, 70)
    y = _dev(np.arange(10, dtype=np.float32))
    x = torch.ones(7, dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(s0, y, x)
    ll = mc.mlem_iterate(s0, y, x, 3, loglik=True)
    assert torch.count_nonzero(x) == 0 and np.all(np.isfinite(ll) | (ll == -np.inf))
    # single event: diagonal 1x1 problem converges in one step
    s1 = mc.mc_system_from_events(3, 2, np.array([1], np.int32), np.array([0], np.int32), 0, 4)
    y = _dev(np.array([0.0, 6.0, 0.0], np.float32))
    x = torch.ones(2, dtype=torch.float32, device="cuda")
    mc.mlem_iterate(s1, y, x, 1)
    # A[1,0] = 1 / n_0 = 1/2  ->  x_0 = y_1 / A = 12
    np.testing.assert_allclose(x.cpu().numpy(), [12.0, 0.0], rtol=1e-6)


@pytest.mark.parametrize("vt", ["f32", "f16", "bf16"])
def test_reduced_precision_values_exact_counts(mc, torso_small, vt):
    # counts stored in half / bfloat16 are exact here: the image equals the
    # FP64 oracle's on the same matrix to the FP32 tolerance
    import torch
    w, pr, a, y, sysm = torso_small
    info = sysm.info()
    limit = {"f32": 1 << 24, "f16": 2048, "bf16": 256}[vt]
    assert info["max_count"] <= limit
    yd = _dev(y)
    sysm.set_value_type(vt)
    x = torch.zeros(pr.n_voxels, dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(sysm, yd, x)
    mc.mlem_iterate(sysm, yd, x, 20)
    sysm.set_value_type("f32")
    want = oracle.mlem(a, y, oracle.mlem_init(a, y), 20)
    assert _rel_l2(x.cpu().numpy(), want) <= MLEM_TOL


def test_half_and_float_values_give_identical_images():
    # short rows (streaming layout): counts <= 2048 are exact in half, the
    # products are formed in float either way and every segment is summed in
    # the same order, so images, log-likelihoods and back-projections must be
    # identical bit for bit
    import torch
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect as mc
    mc.load(B.build())
    w = P.workload("torso64")
    s = mc.mc_build_system(w.phantom, w.geometry, 30_000_000, 3)
    inf = s.info()
    assert inf["spmv_fwd"] == 0 and inf["spmv_bwd"] == 0 and inf["max_count"] <= 2048
    q = torch.zeros(s.shape[0], device="cuda")
    mc.mc_project(s, torch.as_tensor(w.phantom.activity.ravel()).cuda(), q)
    y = torch.as_tensor(P.poisson_counts(q.cpu().numpy(), 1e6, 5)).cuda()
    out = {}
    for vt in ("f32", "f16"):
        s.set_value_type(vt)
        x = torch.zeros(s.shape[1], device="cuda")
        mc.mc_mlem_init(s, y, x)
        ll = mc.mlem_iterate(s, y, x, 7, loglik=True)
        b = torch.zeros(s.shape[1], device="cuda")
        mc.mc_backproject(s, y, b)
        out[vt] = (x.cpu().numpy(), np.asarray(ll), b.cpu().numpy())
    for a, b in zip(out["f32"], out["f16"]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("layout", [0, 4])
def test_loglik_leaves_out_bins_with_an_empty_row(mc, layout):
    # rows 1 and 3 are empty but carry counts (as data from an independent
    # MC realisation does): the likelihood is finite and equals the oracle's
    import torch
    rows = np.array([0, 0, 2, 2, 2, 4], np.int32)
    cols = np.array([0, 1, 1, 2, 2, 0], np.int32)
    s = mc.mc_system_from_events(5, 3, rows, cols, 0, 6)
    mc.mc_system_set_spmv_layout(s, layout, layout)
    c = oracle.system_counts(rows, cols, 5, 3)
    a = oracle.system_matrix(c, oracle.histories_per_voxel(3, 0, 6))
    y = np.array([3.0, 2.0, 5.0, 7.0, 1.0], np.float32)
    x = np.array([1.5, 0.5, 2.0], np.float32)
    v = torch.zeros(1, dtype=torch.float64, device="cuda")
    mc.mc_loglik(s, _dev(x), _dev(y), v)
    want = oracle.loglik(a, x.astype(np.float64), y.astype(np.float64))
    assert np.isfinite(want)
    assert float(v.item()) == pytest.approx(want, rel=1e-6)
    ll = mc.mlem_iterate(s, _dev(y), _dev(x), 4, loglik=True)
    _, llo = oracle.mlem(a, y.astype(np.float64), x.astype(np.float64), 4, with_loglik=True)
    np.testing.assert_allclose(ll, llo, rtol=1e-6)
    s.free()
