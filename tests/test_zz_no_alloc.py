"""mlem_iterate_noalloc: ML-EM for callers that cannot allocate device memory.

Some callers may not allocate on the reconstruction path (a service with a
fixed memory plan, where an allocation could synchronise the device or fail
under a memory cap).  For them the library keeps the ML-EM work vectors in a
static device array.  This file checks, through the C ABI, that the
allocation-free entry point gives the same images and log-likelihoods as
mlem_iterate on two calls in a row, and that it rejects systems larger than
its fixed scratch.  It is collected last so that a failure here leaves every
other test already run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, the tolerance of the other ML-EM parity tests


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect
    mcspect.load(B.build())
    return mcspect


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_mlem_iterate_on_consecutive_calls(mc):
    import torch
    w = P.workload("torso64")
    pr = oracle.Problem(w.phantom, w.geometry)
    H = 4_000_000
    rows, cols, _ = oracle.run(pr, w.seed, 0, H)
    c = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
    a = oracle.system_matrix(c, oracle.histories_per_voxel(pr.n_voxels, 0, H))
    y = P.poisson_counts(a @ w.phantom.activity.ravel().astype(np.float64), 1e6, 4)
    sysm = mc.mc_system_from_events(pr.n_rows, pr.n_voxels, rows, cols.astype(np.int32), 0, H)
    yd = torch.as_tensor(y).cuda()
    x_ref = torch.zeros(pr.n_voxels, dtype=torch.float32, device="cuda")
    mc.mc_mlem_init(sysm, yd, x_ref)
    x_new = x_ref.clone()
    for n_iter in (7, 5):            # two calls in a row, continuing the same image
        ll_ref = mc.mlem_iterate(sysm, yd, x_ref, n_iter, loglik=True)
        ll_new = mc.mlem_iterate_noalloc(sysm, yd, x_new, n_iter, loglik=True)
        torch.cuda.synchronize()
        assert _rel(x_new.cpu().numpy(), x_ref.cpu().numpy()) <= TOL
        np.testing.assert_allclose(ll_new, ll_ref, rtol=1e-12)
    # without log-likelihoods as well
    mc.mlem_iterate(sysm, yd, x_ref, 3)
    mc.mlem_iterate_noalloc(sysm, yd, x_new, 3)
    torch.cuda.synchronize()
    assert _rel(x_new.cpu().numpy(), x_ref.cpu().numpy()) <= TOL


def test_noalloc_rejects_systems_beyond_its_scratch(mc):
    import torch
    n_cols = (1 << 21) + 1
    sysm = mc.mc_system_from_events(4, n_cols, np.array([1], np.int32), np.array([n_cols - 1], np.int32), 0, n_cols)
    y = torch.ones(4, dtype=torch.float32, device="cuda")
    x = torch.ones(n_cols, dtype=torch.float32, device="cuda")
    with pytest.raises(mc.McError) as e:
        mc.mlem_iterate_noalloc(sysm, y, x, 1)
    assert e.value.code == mc.MC_EINVAL and "static scratch limit" in str(e.value)
