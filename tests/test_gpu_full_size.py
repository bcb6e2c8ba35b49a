"""The benchmark's full configuration -- 128^3 torso, 120 views, 10^9
histories in one transport launch, as the benchmark builds it -- checked by
what must hold at any size (paper Sec. 2-3: every history ends in exactly
one fate; Eq. (IMC): C_jv counts events, n_v histories per voxel; Sec. 5.1,
Eq. (MLEM): the update preserves the counts and does not lower the
likelihood) and statistically against the oracle on a sample of the same
workload's histories.  The oracle cannot run 10^9 histories in a test, so
no entry of the full matrix is compared one by one here; the same kernels
are compared entry by entry on smaller ranges in test_gpu_parity.py.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

H = 10 ** 9
# oracle histories for the statistical checks: ten whole passes over the
# 128^3 voxels (history h is emitted in voxel h mod N, so a sample that is
# not a whole number of passes weights some voxels more than others)
SAMPLE = 10 * 128 ** 3


@pytest.fixture(scope="module")
def full():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect as mc
    mc.load(B.build())
    w = P.workload("torso128")
    plan = mc.Plan(w.phantom, w.geometry, "fp32")
    sysm = plan.build(0, H, w.seed)
    cp, ri, cnt, nv = sysm.export_csc()
    rp, ci, cnt_r = sysm.export_csr()
    yield mc, w, sysm, (cp, ri, cnt, nv), (rp, ci, cnt_r)
    sysm.free()
    plan.free()


def test_full_size_tally_invariants(full):
    mc, w, sysm, (cp, ri, cnt, nv), (rp, ci, cnt_r) = full
    inf = sysm.info()
    M, N = inf["n_rows"], inf["n_cols"]
    assert (M, N) == (w.geometry.n_views * w.geometry.n_bins_u * w.geometry.n_bins_v, int(np.prod(w.phantom.shape)))
    assert inf["n_histories"] == H and sum(inf["fates"]) == H      # one fate per history
    assert inf["fates"][3] == 0                                     # no history hit the step cap
    np.testing.assert_array_equal(nv, oracle.histories_per_voxel(N, 0, H))
    assert int(cnt.sum(dtype=np.int64)) == inf["n_events"]          # C_jv counts events
    assert inf["nnz"] == len(ri) and np.all(cnt > 0) and int(cnt.max()) == inf["max_count"]
    # the CSR is the transpose of the CSC, entry for entry
    c_csc = sp.csc_matrix((cnt.astype(np.int64), ri, cp), shape=(M, N))
    c_csr = sp.csr_matrix((cnt_r.astype(np.int64), ci, rp), shape=(M, N))
    assert (c_csc != c_csr).nnz == 0
    # indices strictly increasing within each column and each row
    for ptr, idx in ((cp, ri), (rp, ci)):
        starts = np.zeros(len(idx), bool)
        s = ptr[1:-1]
        starts[s[s < len(idx)]] = True
        assert np.all(np.diff(idx.astype(np.int64))[~starts[1:]] > 0)


def test_full_size_statistics_match_an_oracle_sample(full):
    # fate fractions and events per history over the whole run against the
    # oracle on histories [0, SAMPLE) of the same workload; the bounds are
    # 5 sigma of the sample's binomial / Poisson error (the full run's own
    # error is 50 times smaller)
    mc, w, sysm, (cp, ri, cnt, nv), _ = full
    assert SAMPLE % int(np.prod(w.phantom.shape)) == 0
    pr = oracle.Problem(w.phantom, w.geometry)
    rows, _, fates = oracle.run(pr, w.seed, 0, SAMPLE)
    inf = sysm.info()
    for f in range(3):
        p_orc = int(fates[f]) / SAMPLE
        p_gpu = inf["fates"][f] / H
        assert abs(p_gpu - p_orc) <= 5 * np.sqrt(max(p_orc * (1 - p_orc), 1e-12) / SAMPLE), (f, p_gpu, p_orc)
    # events per history, in all and per group of 15 views (an eighth of
    # the turn): C summed over the group's rows
    g = w.geometry
    per_view = g.n_bins_u * g.n_bins_v
    grp = 15
    c_rows = np.bincount(ri // (per_view * grp), weights=cnt.astype(np.float64), minlength=g.n_views // grp)
    o_rows = np.bincount(rows // (per_view * grp), minlength=g.n_views // grp).astype(np.float64)
    assert len(c_rows) == len(o_rows) == g.n_views // grp
    for tot_g, tot_o in [(c_rows.sum(), o_rows.sum())] + list(zip(c_rows, o_rows)):
        assert abs(tot_g / H - tot_o / SAMPLE) <= 5 * np.sqrt(tot_o) / SAMPLE, (tot_g / H, tot_o / SAMPLE)


def test_full_size_mlem_properties(full):
    # ML-EM on the full matrix through the benchmark's kernels: the
    # sensitivity equals the column sums of C / n_v, the iterates stay
    # non-negative, every update preserves the counts (sum_v s_v x_v =
    # sum_j y_j when every bin with counts has a non-empty row) and the
    # log-likelihood does not decrease
    import torch
    mc, w, sysm, (cp, ri, cnt, nv), (rp, _, _) = full
    M, N = len(rp) - 1, len(cp) - 1
    s = torch.zeros(N, dtype=torch.float64, device="cuda")
    mc.mc_sensitivity(sysm, s)
    s_want = np.zeros(N)
    col_sum = np.bincount(np.repeat(np.arange(N), np.diff(cp)), weights=cnt.astype(np.float64), minlength=N)
    np.divide(col_sum, nv, out=s_want, where=nv > 0)
    s_h = s.cpu().numpy()
    np.testing.assert_allclose(s_h, s_want, rtol=1e-13, atol=0.0)
    reached = np.diff(rp) > 0
    rng = np.random.Generator(np.random.Philox(91))
    y = np.where(reached, rng.poisson(6.0, M), 0).astype(np.float32)
    yd = torch.as_tensor(y).cuda()
    x = torch.zeros(N, dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(sysm, yd, x)
    ll = mc.mlem_iterate(sysm, yd, x, 12, loglik=True)
    xh = x.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(xh)) and np.all(xh >= 0) and np.all(xh[s_h == 0] == 0)
    total = float(y.sum(dtype=np.float64))
    assert abs(float(s_h @ xh) - total) <= 1e-5 * total
    assert np.all(np.diff(ll) >= -1e-7 * np.abs(ll[1:]))
