"""ML-EM through every projector layout and value type, against the FP64
oracle on the same matrix (paper Sec. 5.1, Eq. (MLEM) on the matrix of
Eq. (IMC)), through the C ABI.

The layouts are forced with mc_system_set_spmv_layout: the streaming layout
(warp chunks for short rows, tiles of one warp per row for longer ones), and
row (column) groups of 1..32 lanes.  The matrices are oracle-side count
matrices built from seeded synthetic tallies: long rows and columns (200 to
745 entries per row, as the 10^11-history instance of the 128^3 workload
has), and a short-row matrix of the size of the 128^3, 120-view system.
Value types:
  f32, f16, bf16    -- the counts C_jv, exact at these counts; compared with
                       the oracle on the exact matrix;
  f16_a, bf16_a     -- A = C / n_v rounded to half / bfloat16; compared with
                       the oracle run on that rounded matrix (rounded here
                       with numpy);
and counts above the exact range of half / bfloat16 (allow_rounding): ML-EM
on the rounded counts equals the oracle on that matrix, and its error against
the oracle on the exact matrix stays within the counts' relative rounding.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

MLEM_TOL = 1e-5      # relative L2, FP32 GPU vs FP64 oracle on the same matrix
N_ITER = 20
LAYOUTS = [0, 1, 2, 4, 8, 16, 32]


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    return mcspect


def _rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _round_bf16(a):
    """Round float64 values to the nearest bfloat16 (8 significant bits,
    ties to even), as a double."""
    a = np.asarray(a, np.float64)
    m, e = np.frexp(a)                        # a = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(np.ldexp(m, 8)), e - 8)


def _round_half(a):
    return np.asarray(a, np.float64).astype(np.float16).astype(np.float64)


class _Case:
    """An oracle count matrix from synthetic tallies, its FP64 matrix A, a
    Poisson projection of a smooth image, and the same events on the GPU."""

    def __init__(self, mc, n_rows, n_cols, rows, cols, histories, seed):
        import torch
        self.n_rows, self.n_cols, self.histories = n_rows, n_cols, histories
        self.c = oracle.system_counts(rows, cols, n_rows, n_cols)
        self.n_v = oracle.histories_per_voxel(n_cols, 0, histories)
        self.a = oracle.system_matrix(self.c, self.n_v)
        x_true = 1.0 + 0.5 * np.sin(np.arange(n_cols) * 0.01)
        self.y = P.poisson_counts(self.a @ x_true, 50.0 * n_rows, seed)
        self.yd = torch.as_tensor(self.y).cuda()
        self.sysm = mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, histories)
        self._ref = {}

    def oracle_image(self, a, key="exact"):
        if key not in self._ref:
            self._ref[key] = oracle.mlem(a, self.y, oracle.mlem_init(a, self.y), N_ITER)
        return self._ref[key]

    def a_rounded(self, rnd):
        """A = round(C_jv / n_v) as the rounded-A value types store it."""
        a = sp.csr_matrix(self.c, dtype=np.float64)
        cols = a.indices
        a.data = rnd(a.data / self.n_v[cols].astype(np.float64))
        a.eliminate_zeros()
        return a

    def gpu_image(self, mc):
        import torch
        x = torch.zeros(self.n_cols, dtype=torch.float32, device="cuda")
        mc.mc_mlem_init(self.sysm, self.yd, x)
        mc.mlem_iterate(self.sysm, self.yd, x, N_ITER)
        return x.cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def long_rows(mc):
    # 2048 detector rows x 4096 voxels, rows of 200..745 entries (about 235
    # entries per column), counts 1..3, 3.5 histories per voxel
    n_rows, n_cols = 2048, 4096
    rows, cols = P.random_events(n_rows, n_cols, (200, 745), 3, seed=21)
    return _Case(mc, n_rows, n_cols, rows, cols, int(3.5 * n_cols), seed=22)


def _check_image(got, want, tol=MLEM_TOL):
    assert np.all(np.isfinite(got)) and np.all(got >= 0)
    assert _rel_l2(got, want) <= tol, _rel_l2(got, want)
    # element by element: every voxel within a few float roundings of its
    # share of the image's scale
    scale = float(np.max(np.abs(want)))
    np.testing.assert_allclose(got, want, rtol=2e-4, atol=2e-5 * scale)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("vt", ["f32", "f16", "bf16"])
def test_count_values_every_layout_match_oracle(mc, long_rows, layout, vt):
    case = long_rows
    case.sysm.set_value_type(vt)
    assert mc.mc_system_set_spmv_layout(case.sysm, layout, layout) == (layout, layout)
    want = case.oracle_image(case.a)
    _check_image(case.gpu_image(mc), want)
    case.sysm.set_value_type("f32")


@pytest.mark.parametrize("layout", [0, 4, 32])
@pytest.mark.parametrize("vt,rnd", [("f16_a", _round_half), ("bf16_a", _round_bf16)])
def test_rounded_a_values_match_oracle_on_the_rounded_matrix(mc, long_rows, layout, vt, rnd):
    case = long_rows
    case.sysm.set_value_type(vt)
    assert case.sysm.info()["value_type"] == mc.VALUE_TYPES[vt]
    mc.mc_system_set_spmv_layout(case.sysm, layout, layout)
    a_r = case.a_rounded(rnd)
    want = case.oracle_image(a_r, vt)
    _check_image(case.gpu_image(mc), want)
    # and the rounding is visible against the exact matrix
    assert _rel_l2(case.gpu_image(mc), case.oracle_image(case.a)) > 1e-6
    # the sensitivity is that of the rounded matrix
    import torch
    s = torch.zeros(case.n_cols, dtype=torch.float64, device="cuda")
    mc.mc_sensitivity(case.sysm, s)
    np.testing.assert_allclose(s.cpu().numpy(), oracle.sensitivity(a_r), rtol=1e-12)
    case.sysm.set_value_type("f32")


def test_layout_changes_keep_projections(mc, long_rows):
    import torch
    case = long_rows
    x = torch.as_tensor(np.linspace(0.5, 2.0, case.n_cols).astype(np.float32)).cuda()
    want = case.a @ x.cpu().numpy().astype(np.float64)
    for fwd, bwd in [(0, 32), (8, 0), (-1, 4), (32, -1), (0, 0)]:
        mc.mc_system_set_spmv_layout(case.sysm, fwd, bwd)
        q = torch.zeros(case.n_rows, dtype=torch.float32, device="cuda")
        mc.mc_project(case.sysm, x, q)
        assert _rel_l2(q.cpu().numpy(), want) < 1e-6


def test_layout_rejects_bad_arguments(mc, long_rows):
    with pytest.raises(mc.McError):
        mc.mc_system_set_spmv_layout(long_rows.sysm, 3, 0)
    # a row longer than half a streaming tile cannot be tiled
    n_rows, n_cols = 4, 3000
    rows = np.repeat(np.arange(n_rows, dtype=np.int32), [2500, 10, 10, 10])
    cols = np.concatenate([np.arange(2500), np.arange(10), np.arange(10), np.arange(10)]).astype(np.int32)
    s = mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, n_cols)
    before = s.info()["spmv_fwd"]
    with pytest.raises(mc.McError):
        mc.mc_system_set_spmv_layout(s, 0, -1)
    assert s.info()["spmv_fwd"] == before
    mc.mc_system_set_spmv_layout(s, -1, 0)        # the columns are short: tiles are fine
    assert s.info()["spmv_bwd"] == 0
    s.free()


@pytest.mark.parametrize("vt,count_max,rnd,bound", [("f16", 6000, _round_half, 2.0 ** -10),
                                                     ("bf16", 1000, _round_bf16, 2.0 ** -7)])
def test_counts_beyond_the_exact_range_run_ml_em_on_the_rounded_counts(mc, vt, count_max, rnd, bound):
    # counts up to count_max: half is exact to 2048, bfloat16 to 256.  With
    # allow_rounding the GPU runs ML-EM on the rounded counts (their own
    # column sums as the normaliser): equal to the oracle on that matrix, and
    # within the counts' relative rounding (2^-11, 2^-8; with margin for 20
    # iterations) of the oracle on the exact matrix
    n_rows, n_cols = 128, 256
    rows, cols = P.random_events(n_rows, n_cols, (10, 30), count_max, seed=31)
    case = _Case(mc, n_rows, n_cols, rows, cols, 5 * n_cols, seed=32)
    with pytest.raises(mc.McError):
        case.sysm.set_value_type(vt)                 # not exact: refused by default
    case.sysm.set_value_type(vt, allow_rounding=True)
    got = case.gpu_image(mc)
    c_r = sp.csc_matrix(case.c, dtype=np.float64)
    c_r.data = rnd(c_r.data)
    a_r = oracle.system_matrix(c_r, case.n_v)
    _check_image(got, case.oracle_image(a_r, "rounded counts"))
    err = _rel_l2(got, case.oracle_image(case.a))
    assert 0.0 < err <= bound, err
    case.sysm.free()


def test_mlem_on_a_system_of_the_128_cubed_size_class(mc):
    # 1,966,080 rows (120 views x 128^2 bins) x 2,097,152 voxels and 7.3e6
    # events (rows of ~3.7 entries), as the 10^9-history 128^3 system: the
    # streaming-tile kernels the benchmark runs, and row groups, against the
    # oracle on the same matrix over 50 iterations
    import torch
    n_rows, n_cols = 120 * 128 * 128, 128 ** 3
    rows, cols = P.uniform_events(n_rows, n_cols, 7_300_000, seed=41)
    c = oracle.system_counts(rows, cols, n_rows, n_cols)
    H = 477 * n_cols + 12345
    a = oracle.system_matrix(c, oracle.histories_per_voxel(n_cols, 0, H))
    y = P.poisson_counts(a @ np.ones(n_cols), 2e7, 42)
    want = oracle.mlem(a, y, oracle.mlem_init(a, y), 50)
    sysm = mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, H)
    assert sysm.info()["spmv_fwd"] == 0 and sysm.info()["spmv_bwd"] == 0   # streaming layout (warp chunks) by default
    yd = torch.as_tensor(y).cuda()
    for layout in (0, 4):
        mc.mc_system_set_spmv_layout(sysm, layout, layout)
        x = torch.zeros(n_cols, dtype=torch.float32, device="cuda")
        mc.mc_mlem_init(sysm, yd, x)
        mc.mlem_iterate(sysm, yd, x, 50)
        got = x.cpu().numpy().astype(np.float64)
        assert _rel_l2(got, want) <= MLEM_TOL
        np.testing.assert_allclose(got, want, rtol=1e-4, atol=1e-6 * float(want.max()))
    sysm.free()


@pytest.fixture(scope="module", params=[0.5, 0.2])
def short_rows_ragged(mc, request):
    # short rows and columns (the default streaming layout: warp chunks of
    # 32 R segments, R per lane, entries read in windows of 128) with the
    # awkward cases spelled out: 5013 rows and 3001 columns (the last chunk
    # of either is partial), half (or 80 %) of the rows empty -- rows of
    # ~1.8 (~0.9) entries on average; the launch is too small for more than
    # one row per lane, which the larger cases below cover -- and a run of
    # 512 empty rows (whole empty chunks), one row of 700 entries
    # (several windows), two adjacent rows of 150 entries (window boundaries
    # inside rows), a column of 600 entries and a run of empty columns
    n_rows, n_cols = 5013, 3001
    rows, cols = P.random_events(n_rows, n_cols, (0, 6), 3, seed=51, rows_used=request.param)
    keep = ~((rows >= 1000) & (rows < 1512)) & ~((cols >= 2000) & (cols < 2100))
    rows, cols = rows[keep], cols[keep]
    rng = np.random.Generator(np.random.Philox(52))
    outside = np.setdiff1d(np.arange(n_rows), np.arange(1000, 1512))
    extra_r = [np.full(700, 77), np.full(150, 2015), np.full(150, 2016), rng.choice(outside, 600, replace=False),
               np.array([n_rows - 1])]
    extra_c = [rng.choice(2000, 700, replace=False), rng.choice(2000, 150, replace=False),
               rng.choice(2000, 150, replace=False), np.full(600, 7), np.array([n_cols - 1])]
    rows = np.concatenate([rows] + extra_r).astype(np.int32)
    cols = np.concatenate([cols] + extra_c).astype(np.int32)
    return _Case(mc, n_rows, n_cols, rows, cols, 4 * n_cols + 3, seed=53)


def test_short_segment_layout_edge_cases_match_oracle(mc, short_rows_ragged):
    import torch
    case = short_rows_ragged
    inf = case.sysm.info()
    assert inf["spmv_fwd"] == 0 and inf["spmv_bwd"] == 0
    assert case.c.nnz / case.n_rows < 16 and case.c.nnz / case.n_cols < 16   # warp chunks (not tiles)
    a = case.a.tocsr()
    x = np.linspace(0.5, 2.0, case.n_cols)
    xd = torch.as_tensor(x.astype(np.float32)).cuda()
    q = torch.zeros(case.n_rows, dtype=torch.float32, device="cuda")
    mc.mc_project(case.sysm, xd, q)
    q_want = a @ x.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(q.cpu().numpy(), q_want, rtol=1e-6, atol=1e-7 * q_want.max())
    assert np.all(q.cpu().numpy()[np.diff(a.indptr) == 0] == 0.0)          # empty rows project to 0
    r = np.linspace(0.0, 3.0, case.n_rows)
    b = torch.zeros(case.n_cols, dtype=torch.float32, device="cuda")
    mc.mc_backproject(case.sysm, torch.as_tensor(r.astype(np.float32)).cuda(), b)
    b_want = a.T @ r.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(b.cpu().numpy(), b_want, rtol=1e-6, atol=1e-7 * b_want.max())
    rd = torch.zeros(case.n_rows, dtype=torch.float32, device="cuda")
    mc.mc_project_ratio(case.sysm, xd, case.yd, rd)
    ratio = np.divide(case.y, q_want, out=np.zeros_like(q_want), where=q_want > 0)
    np.testing.assert_allclose(rd.cpu().numpy(), ratio, rtol=1e-5, atol=1e-6 * ratio.max())
    # log-likelihood through the forward kernel's per-block partials
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    mc.mc_loglik(case.sysm, xd, case.yd, ll)
    ll_want = oracle.loglik(a, x.astype(np.float32), case.y)
    assert abs(float(ll[0]) - ll_want) <= 1e-6 * abs(ll_want)
    for vt in ("f32", "f16", "bf16"):
        case.sysm.set_value_type(vt)
        _check_image(case.gpu_image(mc), case.oracle_image(case.a))
    case.sysm.set_value_type("f32")


def _rows_per_lane(nnz, n, launch_segments, sm_count):
    """Rows (columns) per lane that the streaming layout's warp chunks take
    for n segments averaging nnz / n entries in a launch of launch_segments
    segments, restated from the library so that a test can state which
    kernel its case runs."""
    r = 1 if nnz >= 3 * n else 2 if nnz >= 1.5 * n else 4
    while r > 1 and launch_segments // (32 * r) < sm_count * 32:
        r //= 2
    return r


@pytest.mark.parametrize("n_rows,n_cols,n_events,want", [(330_007, 320_009, 640_000, 2),
                                                         (700_001, 650_003, 620_000, 4)])
def test_rows_per_lane_kernels_match_oracle(mc, n_rows, n_cols, n_events, want):
    # systems large enough for the warp chunks to give each lane 2 (4) rows
    # and columns; every projector and ML-EM against the oracle
    import torch
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    rows, cols = P.uniform_events(n_rows, n_cols, n_events, seed=61 + want)
    case = _Case(mc, n_rows, n_cols, rows, cols, 3 * n_cols + 7, seed=62 + want)
    nnz = case.c.nnz
    assert _rows_per_lane(nnz, n_rows, n_rows, sm) == want and _rows_per_lane(nnz, n_cols, n_cols, sm) == want
    inf = case.sysm.info()
    assert inf["spmv_fwd"] == 0 and inf["spmv_bwd"] == 0
    a = case.a.tocsr()
    x = np.linspace(0.5, 2.0, n_cols)
    xd = torch.as_tensor(x.astype(np.float32)).cuda()
    q = torch.zeros(n_rows, dtype=torch.float32, device="cuda")
    mc.mc_project(case.sysm, xd, q)
    q_want = a @ x.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(q.cpu().numpy(), q_want, rtol=1e-6, atol=1e-7 * q_want.max())
    r = np.linspace(0.0, 3.0, n_rows)
    b = torch.zeros(n_cols, dtype=torch.float32, device="cuda")
    mc.mc_backproject(case.sysm, torch.as_tensor(r.astype(np.float32)).cuda(), b)
    b_want = a.T @ r.astype(np.float32).astype(np.float64)
    np.testing.assert_allclose(b.cpu().numpy(), b_want, rtol=1e-6, atol=1e-7 * b_want.max())
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    mc.mc_loglik(case.sysm, xd, case.yd, ll)
    ll_want = oracle.loglik(a, x.astype(np.float32), case.y)
    assert abs(float(ll[0]) - ll_want) <= 1e-6 * abs(ll_want)
    _check_image(case.gpu_image(mc), case.oracle_image(case.a))
    case.sysm.free()
