"""Batched ML-EM (one CUDA graph over many mixed-size systems) and the SpMV
autotuner give the same images as per-system mlem_iterate (through the C
ABI)."""
import numpy as np
import pytest

from paper_2105_13324_gb300 import phantoms as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch_env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2105_13324_gb300 import build as B
    from paper_2105_13324_gb300 import mcspect as mc
    mc.load(B.build())
    mix = P.serving_mix(6, seed=11)
    systems, ys = [], []
    for k, (ph, g, counts, seed) in enumerate(mix):
        s = mc.mc_build_system(ph, g, 3_000_000, seed)
        m, n = s.shape
        q = torch.zeros(m, dtype=torch.float32, device="cuda")
        mc.mc_project(s, torch.as_tensor(ph.activity.ravel()).cuda(), q)
        y = torch.as_tensor(P.poisson_counts(q.cpu().numpy(), counts, seed)).cuda()
        systems.append(s)
        ys.append(y)
    return mc, mix, systems, ys


def _reference(mc, systems, ys, n_iter):
    import torch
    out = []
    for s, y in zip(systems, ys):
        x = torch.zeros(s.shape[1], dtype=torch.float32, device="cuda")
        mc.mc_mlem_init(s, y, x)
        mc.mlem_iterate(s, y, x, n_iter)
        out.append(x.cpu().numpy().astype(np.float64))
    return out


def test_batch_equals_per_system_mlem(batch_env):
    import torch
    mc, mix, systems, ys = batch_env
    xs = [torch.full((s.shape[1],), 7.0, device="cuda") for s in systems]   # overwritten by the start image
    b = mc.Batch(systems, ys, xs)
    ref = _reference(mc, systems, ys, 30)
    for rep in range(2):                       # the captured graph replays identically
        b.mlem(30)
        torch.cuda.synchronize()
        for x, r in zip(xs, ref):
            got = x.cpu().numpy().astype(np.float64)
            assert np.linalg.norm(got - r) / np.linalg.norm(r) < 1e-6
    b.mlem(5)                                  # another iteration count: a second graph
    torch.cuda.synchronize()
    ref5 = _reference(mc, systems, ys, 5)
    for x, r in zip(xs, ref5):
        assert np.linalg.norm(x.cpu().numpy() - r) / np.linalg.norm(r) < 1e-6
    b.free()


def test_autotune_keeps_results(batch_env):
    import torch
    mc, mix, systems, ys = batch_env
    s, y = systems[0], ys[0]
    before = _reference(mc, [s], [y], 10)[0]
    f, bk = mc.mc_system_autotune(s)
    assert f in (0, 1, 2, 4, 8, 16, 32) and bk in (0, 1, 2, 4, 8, 16, 32)
    after = _reference(mc, [s], [y], 10)[0]
    assert np.linalg.norm(after - before) / np.linalg.norm(before) < 1e-5
    ll = mc.mlem_iterate(s, y, torch.ones(s.shape[1], device="cuda"), 3, loglik=True)
    assert np.all(np.isfinite(ll))


def test_batch_after_autotune_and_of_a_forced_detection_system(batch_env):
    # the batch builds its own tiles: systems the autotuner moved to row
    # groups, and weighted (forced-detection) systems, batch like any other
    import torch
    mc, mix, systems, ys = batch_env
    ph, g, counts, seed = mix[1]
    s_fd = mc.mc_build_system(ph, g, 1 << 16, seed, forced=True)
    assert s_fd.info()["weighted"]
    q = torch.zeros(s_fd.shape[0], device="cuda")
    mc.mc_project(s_fd, torch.as_tensor(ph.activity.ravel()).cuda(), q)
    y_fd = torch.as_tensor(P.poisson_counts(q.cpu().numpy(), counts, seed)).cuda()
    s0, y0 = systems[0], ys[0]
    mc.mc_system_autotune(s0)
    ref = _reference(mc, [s0, s_fd], [y0, y_fd], 12)
    xs = [torch.zeros(s.shape[1], device="cuda") for s in (s0, s_fd)]
    b = mc.Batch([s0, s_fd], [y0, y_fd], xs)
    b.mlem(12)
    torch.cuda.synchronize()
    for x, r in zip(xs, ref):
        assert np.linalg.norm(x.cpu().numpy() - r) / np.linalg.norm(r) < 1e-6
    b.free()
