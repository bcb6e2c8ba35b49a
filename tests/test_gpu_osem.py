"""GPU ordered subsets, dual-matrix OS and the additive term vs the oracle
(paper Sec. 5.3-5.4, Eq. (DMOS), Eq. (Sohlberg OSEM)), through the C ABI."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    return mcspect


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_primary_only_matrix_is_bit_exact(mc):
    w = P.workload("water32")
    H = 2_000_000
    g = mc.mc_build_system(w.phantom, w.geometry, H, w.seed, precision="fp64", primary_only=True)
    want = oracle.build_system(oracle.Problem(w.phantom, w.geometry, primary_only=True), w.seed, H)[1]
    cp, ri, cnt, _ = g.export_csc()
    np.testing.assert_array_equal(cp, want.indptr)
    np.testing.assert_array_equal(ri, want.indices)
    np.testing.assert_array_equal(cnt, want.data)


@pytest.fixture(scope="module")
def torso(mc):
    w = P.workload("torso64")
    H = 10_000_000
    out = {}
    for name, prim in (("all", False), ("primary", True)):
        pr = oracle.Problem(w.phantom, w.geometry, primary_only=prim)
        rows, cols, _ = oracle.run(pr, w.seed, 0, H)
        c = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
        a = oracle.system_matrix(c, oracle.histories_per_voxel(pr.n_voxels, 0, H))
        sysm = mc.mc_system_from_events(pr.n_rows, pr.n_voxels, rows, cols.astype(np.int32), 0, H)
        out[name] = (c, a, sysm)
    y = P.poisson_counts(out["all"][1] @ w.phantom.activity.ravel().astype(np.float64), 2e6, 5)
    return w, out, y


def test_subset_systems_are_bit_exact(mc, torso):
    w, out, _ = torso
    c, _, sysm = out["all"]
    rpv = w.geometry.n_bins_u * w.geometry.n_bins_v
    csr = sp.csr_matrix(c)
    for n_sub, s in ((4, 0), (4, 3), (7, 2), (1, 0)):
        sub = mc.mc_system_subset(sysm, rpv, n_sub, s)
        rows = oracle.subset_rows(c.shape[0], rpv, n_sub, s)
        want = sp.csr_matrix(csr[rows])
        want.sort_indices()
        rp, ci, cr = sub.export_csr()
        np.testing.assert_array_equal(rp, want.indptr)
        np.testing.assert_array_equal(ci, want.indices)
        np.testing.assert_array_equal(cr, want.data)
        wc = sp.csc_matrix(want)
        wc.sort_indices()
        cp, ri, cc, nv = sub.export_csc()
        np.testing.assert_array_equal(cp, wc.indptr)
        np.testing.assert_array_equal(ri, wc.indices)
        np.testing.assert_array_equal(cc, wc.data)


@pytest.mark.parametrize("n_sub,dual,with_add", [(1, False, False), (4, False, False), (4, False, True),
                                                  (6, True, False), (6, True, True)])
def test_osem_matches_oracle(mc, torso, n_sub, dual, with_add):
    import torch
    w, out, y = torso
    rpv = w.geometry.n_bins_u * w.geometry.n_bins_v
    _, a_c, s_c = out["all"]
    _, a_b, s_b = out["primary"] if dual else out["all"]
    fwd = [mc.mc_system_subset(s_c, rpv, n_sub, k) if n_sub > 1 else s_c for k in range(n_sub)]
    back = [mc.mc_system_subset(s_b, rpv, n_sub, k) if n_sub > 1 else s_b for k in range(n_sub)]
    add = None
    if with_add:
        add = (0.3 * (a_c @ np.ones(a_c.shape[1])) + 0.05).astype(np.float32)
    x0 = oracle.mlem_init(a_c, y).astype(np.float32)
    x = torch.as_tensor(x0).cuda()
    yd = torch.as_tensor(y).cuda()
    mc.osem_iterate(fwd, back, yd, x, 4, add=torch.as_tensor(add).cuda() if with_add else None)
    subsets = [oracle.subset_rows(a_c.shape[0], rpv, n_sub, k) for k in range(n_sub)]
    want = oracle.osem(a_c, a_b, subsets, y, x0.astype(np.float64), 4, add=add)
    assert _rel(x.cpu().numpy(), want) <= TOL
    if n_sub == 1 and not dual and not with_add:
        x2 = torch.as_tensor(x0).cuda()
        mc.mlem_iterate(s_c, yd, x2, 4)
        assert _rel(x.cpu().numpy(), x2.cpu().numpy().astype(np.float64)) <= 1e-6


def test_osem_rejects_mismatched_subsets(mc, torso):
    import torch
    w, out, y = torso
    rpv = w.geometry.n_bins_u * w.geometry.n_bins_v
    s_c = out["all"][2]
    a = [mc.mc_system_subset(s_c, rpv, 2, k) for k in range(2)]
    x = torch.ones(s_c.shape[1], device="cuda")
    with pytest.raises(mc.McError):
        mc.osem_iterate(a, [a[1], a[0]], torch.as_tensor(y).cuda(), x, 1)
