"""Batched ML-EM (one CUDA graph over many mixed-size systems) and the SpMV
autotuner against the FP64 oracle (paper Sec. 5.1, Eq. (MLEM)), through the
C ABI.

Every system is the oracle's own tally of a serving-mix acquisition (48^3 to
128^3 grids, 40 to 120 views), handed to the library as an event list, so
the batched images are compared with oracle.mlem on the same matrix and
projections.
"""
import numpy as np
import pytest

import oracle
from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu

MLEM_TOL = 1e-5     # relative L2, FP32 GPU vs FP64 oracle on the same matrix
HISTORIES = 3_000_000


def _rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def batch_env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect as mc
    mc.load(B.build())
    mix = P.serving_mix(6, seed=11)
    systems, ys, cases = [], [], []
    for ph, g, counts, seed in mix:
        pr = oracle.Problem(ph, g)
        rows, cols, _ = oracle.run(pr, seed, 0, HISTORIES)
        c = oracle.system_counts(rows, cols, pr.n_rows, pr.n_voxels)
        a = oracle.system_matrix(c, oracle.histories_per_voxel(pr.n_voxels, 0, HISTORIES))
        y = P.poisson_counts(a @ ph.activity.ravel().astype(np.float64), counts, seed)
        systems.append(mc.mc_system_from_events(pr.n_rows, pr.n_voxels, rows, cols, 0, HISTORIES))
        ys.append(torch.as_tensor(y).cuda())
        cases.append((a, y))
    return mc, mix, systems, ys, cases


def _oracle_images(cases, n_iter):
    return [oracle.mlem(a, y, oracle.mlem_init(a, y), n_iter) for a, y in cases]


def test_batch_equals_oracle_mlem(batch_env):
    import torch
    mc, mix, systems, ys, cases = batch_env
    xs = [torch.full((s.shape[1],), 7.0, device="cuda") for s in systems]   # overwritten by the start image
    b = mc.Batch(systems, ys, xs)
    want = _oracle_images(cases, 30)
    for rep in range(2):                       # the captured graph replays identically
        b.mlem(30)
        torch.cuda.synchronize()
        for x, w in zip(xs, want):
            assert _rel_l2(x.cpu().numpy(), w) <= MLEM_TOL
    b.mlem(5)                                  # another iteration count: a second graph
    torch.cuda.synchronize()
    for x, w in zip(xs, _oracle_images(cases, 5)):
        got = x.cpu().numpy().astype(np.float64)
        assert _rel_l2(got, w) <= MLEM_TOL
        np.testing.assert_allclose(got, w, rtol=1e-4, atol=1e-6 * float(w.max()))
    b.free()


def test_persistent_batch_equals_oracle_mlem(batch_env):
    # all iterations in one cooperative launch: the same images
    import torch
    mc, mix, systems, ys, cases = batch_env
    xs = [torch.full((s.shape[1],), 3.0, device="cuda") for s in systems]
    b = mc.Batch(systems, ys, xs)
    for n_iter in (30, 1, 0):
        b.mlem_persistent(n_iter)
        torch.cuda.synchronize()
        want = _oracle_images(cases, n_iter)
        for x, w in zip(xs, want):
            got = x.cpu().numpy().astype(np.float64)
            assert _rel_l2(got, w) <= MLEM_TOL
    b.free()


def test_autotune_keeps_results(batch_env):
    import torch
    mc, mix, systems, ys, cases = batch_env
    s, y = systems[0], ys[0]
    want = _oracle_images(cases[:1], 10)[0]
    f, bk = mc.mc_system_autotune(s)
    assert f in (0, 1, 2, 4, 8, 16, 32) and bk in (0, 1, 2, 4, 8, 16, 32)
    x = torch.zeros(s.shape[1], device="cuda")
    mc.mc_mlem_init(s, y, x)
    mc.mlem_iterate(s, y, x, 10)
    assert _rel_l2(x.cpu().numpy(), want) <= MLEM_TOL
    ll = mc.mlem_iterate(s, y, torch.ones(s.shape[1], device="cuda"), 3, loglik=True)
    assert np.all(np.isfinite(ll))


def test_batch_after_autotune_and_of_a_forced_detection_system(batch_env):
    # the batch builds its own tiles: systems the autotuner moved to row
    # groups, and weighted (forced-detection) systems, batch like any other
    import torch
    mc, mix, systems, ys, cases = batch_env
    ph, g, counts, seed = mix[1]
    H = 1 << 14
    pr = oracle.Problem(ph, g, forced_detection=True)
    rows, cols, q, _ = oracle.run_fd(pr, seed, 0, H)
    w = oracle.system_weights(rows, cols, q, pr.n_rows, pr.n_voxels)
    a_fd = oracle.system_matrix(w, oracle.histories_per_voxel(pr.n_voxels, 0, H))
    y_fd = P.poisson_counts(a_fd @ ph.activity.ravel().astype(np.float64), counts, seed)
    s_fd = mc.mc_system_from_weighted_events(pr.n_rows, pr.n_voxels, rows, cols, q.astype(np.uint64), 0, H)
    assert s_fd.info()["weighted"]
    s0, y0 = systems[0], ys[0]
    mc.mc_system_autotune(s0)
    want = _oracle_images([cases[0], (a_fd, y_fd)], 12)
    xs = [torch.zeros(s.shape[1], device="cuda") for s in (s0, s_fd)]
    b = mc.Batch([s0, s_fd], [y0, torch.as_tensor(y_fd).cuda()], xs)
    b.mlem(12)
    torch.cuda.synchronize()
    for x, wi in zip(xs, want):
        assert _rel_l2(x.cpu().numpy(), wi) <= MLEM_TOL
    b.free()
    s_fd.free()


def test_batch_with_four_rows_per_lane_equals_oracle_mlem(batch_env):
    # three systems whose non-empty rows and columns average ~1.2 entries,
    # together large enough for the batch's warp chunks to give each lane 4
    # rows (columns); graph and cooperative forms against oracle.mlem
    import torch
    mc = batch_env[0]
    n_rows, n_cols = 700_001, 650_003
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    systems, ys, cases = [], [], []
    m_all = n_all = 0
    for k in range(3):
        rows, cols = P.uniform_events(n_rows, n_cols, 300_000, seed=71 + k)
        c = oracle.system_counts(rows, cols, n_rows, n_cols)
        H = 2 * n_cols + 1000 * k
        a = oracle.system_matrix(c, oracle.histories_per_voxel(n_cols, 0, H))
        y = P.poisson_counts(a @ np.ones(n_cols), 2e5, 81 + k)
        m_c = int(np.count_nonzero(np.diff(c.tocsr().indptr)))
        n_c = int(np.count_nonzero(np.diff(c.tocsc().indptr)))
        assert c.nnz < 1.5 * m_c and c.nnz < 1.5 * n_c
        m_all, n_all = m_all + m_c, n_all + n_c
        systems.append(mc.mc_system_from_events(n_rows, n_cols, rows, cols, 0, H))
        ys.append(torch.as_tensor(y).cuda())
        cases.append((a, y))
    assert m_all // 128 >= 32 * sm and n_all // 128 >= 32 * sm   # 4 rows per lane
    xs = [torch.zeros(n_cols, device="cuda") for _ in systems]
    b = mc.Batch(systems, ys, xs)
    want = _oracle_images(cases, 15)
    for run in (b.mlem, b.mlem_persistent):
        run(15)
        torch.cuda.synchronize()
        for x, w in zip(xs, want):
            got = x.cpu().numpy().astype(np.float64)
            assert _rel_l2(got, w) <= MLEM_TOL
            np.testing.assert_allclose(got, w, rtol=1e-4, atol=1e-6 * float(w.max()))
    b.free()
    for s in systems:
        s.free()
